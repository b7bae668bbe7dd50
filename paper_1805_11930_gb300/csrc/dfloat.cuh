// Double-float ("double-word") arithmetic: a value is the unevaluated sum of
// two FP32 numbers h + l with |l| <= ulp(h)/2, about 48 significant bits.
//
// On GB300 the FP64 pipe issues 1/62 of the FP32 rate, so an operator whose
// FP64 accuracy matters but whose work is FMA chains runs faster on FP32 pairs.
// Built from the classical error-free transformations:
//   TwoSum (Knuth):       s = a + b exactly as s_h + s_l, 6 additions;
//   Fast2Sum (Dekker):    the same for |a| >= |b|, 3 additions;
//   TwoProd with an FMA:  a b = p + e, p = a*b, e = fma(a, b, -p), exact.
// Sums use the "sloppy" double-word addition (TwoSum of the high parts, the
// low parts added in FP32, one Fast2Sum to renormalise): its error is a few
// 2^-48 times |x| + |y|, the same form as the rounding of an FP64 addition;
// products add the two cross terms to the exact product of the high parts.
// Scalars that need a quotient or a square root go through FP64 (few per cell).
#pragma once

#include <cuda_runtime.h>

namespace dgmg {

struct df {
  float h, l;
  df() = default;   // trivial, so that df can live in __constant__ memory
  __host__ __device__ df(int v) : h((float)v), l(0.f) {}
  __host__ __device__ df(float v) : h(v), l(0.f) {}
  __host__ __device__ df(float hi, float lo) : h(hi), l(lo) {}
  __host__ __device__ explicit df(double v) {
    h = (float)v;
    l = (float)(v - (double)h);
  }
  __host__ __device__ explicit operator double() const { return (double)h + (double)l; }
};

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  const float s = a + b;
  return df(s, b - (s - a));
}

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  return df(s, (a - (s - bb)) + (b - bb));
}

__device__ __forceinline__ df operator+(df x, df y) {
  const df s = two_sum(x.h, y.h);
  return fast_two_sum(s.h, s.l + (x.l + y.l));
}

__device__ __forceinline__ df operator-(df x) { return df(-x.h, -x.l); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }

__device__ __forceinline__ df operator*(df x, df y) {
  const float p = x.h * y.h;
  float e = fmaf(x.h, y.h, -p);
  e = fmaf(x.h, y.l, e);
  e = fmaf(x.l, y.h, e);
  return fast_two_sum(p, e);
}

// x * y + z with one renormalisation.
__device__ __forceinline__ df fma(df x, df y, df z) {
  const float p = x.h * y.h;
  float e = fmaf(x.h, y.h, -p);
  e = fmaf(x.h, y.l, e);
  e = fmaf(x.l, y.h, e);
  const df s = two_sum(p, z.h);
  return fast_two_sum(s.h, s.l + (e + z.l));
}

__device__ __forceinline__ df& operator+=(df& x, df y) {
  x = x + y;
  return x;
}
__device__ __forceinline__ df& operator*=(df& x, df y) {
  x = x * y;
  return x;
}

// Comparisons on normalised pairs: the high part decides unless it is equal.
__device__ __forceinline__ bool operator<=(df x, df y) { return x.h < y.h || (x.h == y.h && x.l <= y.l); }
__device__ __forceinline__ bool operator>(df x, df y) { return !(x <= y); }
__device__ __forceinline__ bool operator>=(df x, df y) { return x.h > y.h || (x.h == y.h && x.l >= y.l); }
__device__ __forceinline__ bool operator<(df x, df y) { return !(x >= y); }
__device__ __forceinline__ bool operator!=(df x, df y) { return x.h != y.h || x.l != y.l; }

__device__ __forceinline__ df sqrt(df x) { return df(::sqrt((double)x)); }
__device__ __forceinline__ df fabs(df x) { return x.h < 0.f || (x.h == 0.f && x.l < 0.f) ? -x : x; }
__device__ __forceinline__ df hypot(df a, df b) { return df(::hypot((double)a, (double)b)); }
__device__ __forceinline__ df operator/(df a, df b) { return df((double)a / (double)b); }

// The float / double overloads stay visible next to the df ones.
using ::fabs;
using ::fma;
using ::hypot;
using ::sqrt;

// Dot product sum_j a_j x_j of n double-float pairs with one renormalisation:
// the high parts are summed with TwoSum, all low-order terms (the product
// errors, the cross terms a.h x.l + a.l x.h and the TwoSum errors) in one FP32
// accumulator; 12 FP32 operations per term instead of 15 for a chain of fma.
struct df_acc {
  float sh, c;
  __device__ __forceinline__ df_acc() : sh(0.f), c(0.f) {}
  __device__ __forceinline__ void add_prod(df a, df x) {
    const float p = a.h * x.h;
    c += fmaf(a.h, x.h, -p);
    c = fmaf(a.h, x.l, c);
    c = fmaf(a.l, x.h, c);
    const float s = sh + p;
    const float bb = s - sh;
    c += (sh - (s - bb)) + (p - bb);
    sh = s;
  }
  __device__ __forceinline__ df value() const { return two_sum(sh, c); }   // exact even if |c| > |sh|
};

__device__ __forceinline__ df shfl_xor(df v, int o) {
  return df(__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o));
}

}  // namespace dgmg
