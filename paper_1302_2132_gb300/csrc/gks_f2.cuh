// Two single-precision lanes in one register pair (sm_100 and later): the flux of two faces evaluated
// by one thread with the paired FP32 instructions (FFMA2, FMUL2, FADD2), one issue slot for two
// operations.  F2 carries the two faces' values; products are kept as a pending (a, b) pair so that
// a * b + c becomes one fused multiply-add, as the compiler would contract it for scalars.
#pragma once
#ifndef GKS_HOST_COUNT
#include <cuda_runtime.h>
#define GKS_F2FN __device__ __forceinline__
#else
#include <math.h>
#define GKS_F2FN inline
#endif

namespace gks {

#ifdef GKS_HOST_COUNT
// Host form, for the test harnesses that compile the flux for the CPU: a plain pair of floats, and
// the paired operations as per-lane fused multiply-add, product and sum, each rounded once as the
// paired instructions round each lane.
struct float2 {
  float x, y;
};
inline float2 make_float2(float a, float b) { return float2{a, b}; }
#endif

struct F2 {
  float2 v;
  F2() = default;
  GKS_F2FN F2(float a) : v(make_float2(a, a)) {}
  GKS_F2FN F2(double a) : v(make_float2((float)a, (float)a)) {}
  GKS_F2FN F2(int a) : v(make_float2((float)a, (float)a)) {}
  GKS_F2FN F2(float a, float b) : v(make_float2(a, b)) {}
  GKS_F2FN explicit F2(float2 a) : v(a) {}
};

#ifndef GKS_HOST_COUNT
GKS_F2FN F2 f2_fma(F2 a, F2 b, F2 c) { return F2(__ffma2_rn(a.v, b.v, c.v)); }
GKS_F2FN F2 f2_mul(F2 a, F2 b) { return F2(__fmul2_rn(a.v, b.v)); }
GKS_F2FN F2 f2_add(F2 a, F2 b) { return F2(__fadd2_rn(a.v, b.v)); }
#else
inline F2 f2_fma(F2 a, F2 b, F2 c) { return F2(fmaf(a.v.x, b.v.x, c.v.x), fmaf(a.v.y, b.v.y, c.v.y)); }
inline F2 f2_mul(F2 a, F2 b) { return F2(a.v.x * b.v.x, a.v.y * b.v.y); }
inline F2 f2_add(F2 a, F2 b) { return F2(a.v.x + b.v.x, a.v.y + b.v.y); }
#endif
GKS_F2FN F2 f2_neg(F2 a) { return F2(make_float2(-a.v.x, -a.v.y)); }

// a pending product a * b: consumed by + and - as one fused multiply-add, else rounded as a product
struct F2Mul {
  F2 a, b;
  GKS_F2FN operator F2() const { return f2_mul(a, b); }
};

GKS_F2FN F2Mul operator*(F2 a, F2 b) { return F2Mul{a, b}; }
GKS_F2FN F2Mul operator*(F2Mul m, F2 b) { return F2Mul{F2(m), b}; }
GKS_F2FN F2Mul operator*(F2 a, F2Mul m) { return F2Mul{a, F2(m)}; }
GKS_F2FN F2Mul operator*(F2Mul m, F2Mul n) { return F2Mul{F2(m), F2(n)}; }
GKS_F2FN F2 operator+(F2 a, F2 b) { return f2_add(a, b); }
GKS_F2FN F2 operator+(F2Mul m, F2 c) { return f2_fma(m.a, m.b, c); }
GKS_F2FN F2 operator+(F2 c, F2Mul m) { return f2_fma(m.a, m.b, c); }
GKS_F2FN F2 operator+(F2Mul m, F2Mul n) { return f2_fma(m.a, m.b, F2(n)); }
GKS_F2FN F2 operator-(F2 a) { return f2_neg(a); }
GKS_F2FN F2Mul operator-(F2Mul m) { return F2Mul{f2_neg(m.a), m.b}; }
GKS_F2FN F2 operator-(F2 a, F2 b) { return f2_add(a, f2_neg(b)); }
GKS_F2FN F2 operator-(F2 c, F2Mul m) { return f2_fma(f2_neg(m.a), m.b, c); }
GKS_F2FN F2 operator-(F2Mul m, F2 c) { return f2_fma(m.a, m.b, f2_neg(c)); }
GKS_F2FN F2 operator-(F2Mul m, F2Mul n) { return f2_fma(m.a, m.b, f2_neg(F2(n))); }
GKS_F2FN F2& operator+=(F2& a, F2 b) { return a = a + b; }
GKS_F2FN F2& operator+=(F2& a, F2Mul m) { return a = a + m; }
GKS_F2FN F2& operator-=(F2& a, F2 b) { return a = a - b; }
GKS_F2FN F2& operator-=(F2& a, F2Mul m) { return a = a - m; }
GKS_F2FN F2& operator*=(F2& a, F2 b) { return a = F2(a * b); }

}  // namespace gks
