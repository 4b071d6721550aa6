// Static operation count of the interface flux: the device flux code of gks_flux.cuh is compiled
// for the host with a scalar type that counts every arithmetic operation it performs.  Operations
// whose operand is a literal 0 or 1 are not counted (the compiler removes them), so the count is
// that of the algorithm as written.  Used for the algorithmic FLOP figure of the roofline.
#define GKS_HOST_COUNT 1
#define GKS_FN inline
#include <cmath>
#include <cstring>

namespace gks {
struct Cnt;
}
#include "gks_flux.cuh"

namespace gks {

struct Ops {
  long long add, mul, div, sqrt, exp, erfc;
};
static thread_local Ops g_ops;

// k: 0 value computed at run time, 1 literal zero, 2 literal one, 3 other literal
struct Cnt {
  double v;
  int k;
  Cnt() : v(0.0), k(1) {}
  Cnt(double x) : v(x), k(x == 0.0 ? 1 : (x == 1.0 ? 2 : 3)) {}
  Cnt(int x) : Cnt((double)x) {}
  static Cnt run(double x) {
    Cnt c;
    c.v = x;
    c.k = 0;
    return c;
  }
  explicit operator double() const { return v; }
};
inline bool lit(const Cnt& a) { return a.k != 0; }
inline Cnt operator+(const Cnt& a, const Cnt& b) {
  if (a.k == 1) return b;
  if (b.k == 1) return a;
  if (lit(a) && lit(b)) return Cnt(a.v + b.v);
  g_ops.add++;
  return Cnt::run(a.v + b.v);
}
inline Cnt operator-(const Cnt& a, const Cnt& b) {
  if (b.k == 1) return a;
  if (lit(a) && lit(b)) return Cnt(a.v - b.v);
  g_ops.add++;
  return Cnt::run(a.v - b.v);
}
inline Cnt operator-(const Cnt& a) { return lit(a) ? Cnt(-a.v) : Cnt::run(-a.v); }
inline Cnt operator*(const Cnt& a, const Cnt& b) {
  if (a.k == 1 || b.k == 1) return Cnt(0.0);
  if (a.k == 2) return b;
  if (b.k == 2) return a;
  if (lit(a) && lit(b)) return Cnt(a.v * b.v);
  g_ops.mul++;
  return Cnt::run(a.v * b.v);
}
inline Cnt operator/(const Cnt& a, const Cnt& b) {
  if (b.k == 2) return a;
  if (lit(a) && lit(b)) return Cnt(a.v / b.v);
  g_ops.div++;
  return Cnt::run(a.v / b.v);
}
inline Cnt& operator+=(Cnt& a, const Cnt& b) { return a = a + b; }
inline Cnt& operator-=(Cnt& a, const Cnt& b) { return a = a - b; }
inline Cnt& operator*=(Cnt& a, const Cnt& b) { return a = a * b; }
inline bool operator<(const Cnt& a, const Cnt& b) { return a.v < b.v; }
inline bool operator>(const Cnt& a, const Cnt& b) { return a.v > b.v; }

template <> inline Cnt g_sqrt<Cnt>(Cnt x) {
  g_ops.sqrt++;
  return Cnt::run(std::sqrt(x.v));
}
template <> inline Cnt g_exp<Cnt>(Cnt x) {
  g_ops.exp++;
  return Cnt::run(std::exp(x.v));
}
template <> inline Cnt g_erfc<Cnt>(Cnt x) {
  g_ops.erfc++;
  return Cnt::run(std::erfc(x.v));
}

template <int D, bool M>
static void count_face(int with_recon, Ops* out) {
  constexpr int nv = D + 2;
  g_ops = Ops{0, 0, 0, 0, 0, 0};
  // a representative face: distinct positive states, dt/tau > 1 (the closed-form time branch)
  Cnt s[4][nv], wl[nv], wr[nv], cl[nv], cr[nv], sl[nv], sr[nv], tl[Dims<D>::nt][nv], tr[Dims<D>::nt][nv];
  for (int c = 0; c < 4; ++c)
    for (int v = 0; v < nv; ++v) s[c][v] = Cnt::run(v == 0 ? 1.0 + 0.1 * c : (v == nv - 1 ? 2.5 + 0.2 * c : 0.1 * (c + v)));
  const Cnt h = Cnt::run(0.01);
  // the step kernel reads the limited cell slopes from shared memory (computed once per cell, see
  // count_cell) and forms the face values w = W +- (h/2) s
  for (int v = 0; v < nv; ++v) {
    sl[v] = Cnt::run(0.3);
    sr[v] = Cnt::run(0.2);
    if (with_recon) {
      wl[v] = s[1][v] + Cnt(0.5) * h * sl[v];
      wr[v] = s[2][v] - Cnt(0.5) * h * sr[v];
    } else {
      wl[v] = s[1][v];
      wr[v] = s[2][v];
    }
    cl[v] = s[1][v];
    cr[v] = s[2][v];
    for (int t = 0; t < Dims<D>::nt; ++t) {
      tl[t][v] = M ? Cnt::run(0.1) : Cnt(0.0);
      tr[t][v] = M ? Cnt::run(0.1) : Cnt(0.0);
    }
  }
  Gas<Cnt> gas;
  gas.bK = Cnt::run(5.0);
  gas.ibK = Cnt::run(0.2);
  gas.K = Cnt::run(5.0 - D);
  gas.mu = Cnt::run(1e-5);
  gas.C_a = Cnt::run(0.0);
  Cnt F[nv], tau;
  face_flux<D, Cnt, M>(wl, wr, cl, cr, sl, sr, tl, tr, Cnt::run(0.005), Cnt::run(0.005), Cnt::run(1e-5),
                       Cnt::run(1e-3), gas, 0, F, &tau);
  *out = g_ops;
}

// Per cell of the step: the van Leer-limited slope of every variable along every axis (two
// differences times the tabulated inverse centre distances, the limiter), done once per cell and
// axis.  The inverse distances are computed once per tile row and are not counted.
template <int D>
static void count_cell(Ops* out) {
  constexpr int nv = D + 2;
  g_ops = Ops{0, 0, 0, 0, 0, 0};
  for (int a = 0; a < D; ++a) {
    const Cnt im = Cnt::run(100.0), ip = Cnt::run(90.0);
    for (int v = 0; v < nv; ++v) {
      const Cnt cm = Cnt::run(1.0), c0 = Cnt::run(1.1), cp = Cnt::run(1.3);
      (void)limiter<Cnt>(LIM_VANLEER, (c0 - cm) * im, (cp - c0) * ip);
    }
  }
  *out = g_ops;
}

// Per face of a higher-order reconstruction: the face values of both sides for every variable
// (recon 1: third-order MUSCL, 2: fifth-order WENO) and the two one-sided normal slopes.
template <int D>
static void count_recon(int recon, Ops* out) {
  constexpr int nv = D + 2;
  g_ops = Ops{0, 0, 0, 0, 0, 0};
  const Cnt i2h = Cnt::run(200.0);
  for (int v = 0; v < nv; ++v) {
    const Cnt a = Cnt::run(1.0), b = Cnt::run(1.1), c = Cnt::run(1.3), d = Cnt::run(1.4), e = Cnt::run(1.6),
              f = Cnt::run(1.65);
    Cnt wl, wr;
    if (recon == 2) {
      wl = weno5<Cnt>(a, b, c, d, e);
      wr = weno5<Cnt>(f, e, d, c, b);
    } else {
      wl = muscl3_right<Cnt>(b, c, d);
      wr = muscl3_left<Cnt>(c, d, e);
    }
    (void)((wl - c) * i2h);
    (void)((d - wr) * i2h);
  }
  *out = g_ops;
}

}  // namespace gks

extern "C" int gks_recon_op_count(int dim, int recon, long long* counts) {
  gks::Ops o{0, 0, 0, 0, 0, 0};
  if (recon != 1 && recon != 2) return 1;
  if (dim == 1)
    gks::count_recon<1>(recon, &o);
  else if (dim == 2)
    gks::count_recon<2>(recon, &o);
  else if (dim == 3)
    gks::count_recon<3>(recon, &o);
  else
    return 1;
  counts[0] = o.add;
  counts[1] = o.mul;
  counts[2] = o.div;
  counts[3] = o.sqrt;
  counts[4] = o.exp;
  counts[5] = o.erfc;
  return 0;
}

extern "C" int gks_cell_op_count(int dim, long long* counts) {
  gks::Ops o{0, 0, 0, 0, 0, 0};
  if (dim == 1)
    gks::count_cell<1>(&o);
  else if (dim == 2)
    gks::count_cell<2>(&o);
  else if (dim == 3)
    gks::count_cell<3>(&o);
  else
    return 1;
  counts[0] = o.add;
  counts[1] = o.mul;
  counts[2] = o.div;
  counts[3] = o.sqrt;
  counts[4] = o.exp;
  counts[5] = o.erfc;
  return 0;
}

extern "C" int gks_face_op_count(int dim, int expand, int with_recon, long long* counts) {
  gks::Ops o{0, 0, 0, 0, 0, 0};
  if (dim == 1)
    gks::count_face<1, false>(with_recon, &o);
  else if (dim == 2 && expand)
    gks::count_face<2, true>(with_recon, &o);
  else if (dim == 2)
    gks::count_face<2, false>(with_recon, &o);
  else if (dim == 3 && expand)
    gks::count_face<3, true>(with_recon, &o);
  else if (dim == 3)
    gks::count_face<3, false>(with_recon, &o);
  else
    return 1;
  counts[0] = o.add;
  counts[1] = o.mul;
  counts[2] = o.div;
  counts[3] = o.sqrt;
  counts[4] = o.exp;
  counts[5] = o.erfc;
  return 0;
}
