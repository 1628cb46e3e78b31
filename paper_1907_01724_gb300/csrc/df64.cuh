// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi)/2), giving about 46 significant bits on the FP32 pipes.  Built from the
// error-free transformations of Knuth (two-sum), Dekker (fast two-sum) and the FMA form of
// Dekker's exact product; on this GPU FP64 arithmetic runs at about 1/73 of FP32, so these
// sequences of 5-10 FP32 operations are several times faster than one FP64 operation.
// Operations here never change rounding-sensitive order: the compiler does not reassociate
// FP32 sums, and every product whose rounding error is needed is an explicit fmaf.
#pragma once

#include <cuda_runtime.h>

namespace hsma {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo)
{
  df r;
  r.hi = hi;
  r.lo = lo;
  return r;
}

// exact: a + b = s + e (Knuth)
__device__ __forceinline__ df two_sum(float a, float b)
{
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return df_make(s, e);
}

// exact when |a| >= |b| (Dekker)
__device__ __forceinline__ df fast_two_sum(float a, float b)
{
  const float s = a + b;
  return df_make(s, b - (s - a));
}

// exact: a * b = p + e
__device__ __forceinline__ df two_prod(float a, float b)
{
  const float p = a * b;
  return df_make(p, fmaf(a, b, -p));
}

__device__ __forceinline__ df df_from_double(double x)
{
  const float hi = __double2float_rn(x);
  return df_make(hi, __double2float_rn(x - (double)hi));
}

__device__ __forceinline__ double df_to_double(df x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ df operator+(df x, df y)
{
  df s = two_sum(x.hi, y.hi);
  s.lo += x.lo + y.lo;
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df operator-(df x) { return df_make(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }

__device__ __forceinline__ df operator*(df x, df y)
{
  df p = two_prod(x.hi, y.hi);
  p.lo = fmaf(x.hi, y.lo, p.lo);
  p.lo = fmaf(x.lo, y.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

// x * y + z
__device__ __forceinline__ df df_fma(df x, df y, df z) { return x * y + z; }

// a x - b y with a single renormalisation: the two leading products and their exact errors
// (FMA form), the difference of the leading products as an exact two-sum, the four cross
// terms folded into the low part.  ~19 FP32 operations against ~25 for two products and a sum.
__device__ __forceinline__ df df_mul_sub(df a, df x, df b, df y)
{
  const float p1 = a.hi * x.hi;
  const float e1 = fmaf(a.hi, x.hi, -p1);
  const float p2 = b.hi * y.hi;
  const float e2 = fmaf(b.hi, y.hi, -p2);
  const df s = two_sum(p1, -p2);
  float lo = s.lo + (e1 - e2);
  lo = fmaf(a.hi, x.lo, lo);
  lo = fmaf(a.lo, x.hi, lo);
  lo = fmaf(-b.hi, y.lo, lo);
  lo = fmaf(-b.lo, y.hi, lo);
  return fast_two_sum(s.hi, lo);
}

// acc + a b without renormalising the accumulator: the rounding error of the high-part sum
// (two-sum) and of the product (FMA form and cross terms) go to the low part, which stays
// ~2^-24 of the high part over a few dozen terms; df_norm renormalises once at the end.
__device__ __forceinline__ df df_acc(df acc, df a, df b)
{
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  const df s = two_sum(acc.hi, p);
  return df_make(s.hi, acc.lo + (s.lo + e));
}

__device__ __forceinline__ df df_norm(df x) { return fast_two_sum(x.hi, x.lo); }

// 1/b: the correctly rounded FP32 reciprocal of the high part, then one Newton step for
// f(y) = 1/y - b in double-float, y <- y + y (1 - b y), which squares the 2^-24 relative error.
__device__ __forceinline__ df df_recip(df b)
{
  const float y = __frcp_rn(b.hi);
  const df yd = df_make(y, 0.f);
  const df e = df_make(1.f, 0.f) - b * yd;
  return yd + e * yd;
}

// sqrt(a), a > 0: the FP32 square root of the high part, then one Newton (Heron) step in
// double-float, s <- s + (a - s^2) / (2 s).
__device__ __forceinline__ df df_sqrt(df a)
{
  const float s = sqrtf(a.hi);
  const df sd = df_make(s, 0.f);
  const df r = a - two_prod(s, s);
  return sd + r * df_make(0.5f / s, 0.f);
}

}  // namespace hsma
