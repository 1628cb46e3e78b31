// Double-float arithmetic: a value is an unevaluated sum hi + lo of two FP32 numbers
// (|lo| <= ulp(hi)/2), giving about 46 significant bits on the FP32 pipes.  Built from the
// error-free transformations of Knuth (two-sum), Dekker (fast two-sum) and the FMA form of
// Dekker's exact product; on this GPU FP64 arithmetic runs at about 1/73 of FP32, so these
// sequences of 5-10 FP32 operations are several times faster than one FP64 operation.
// Operations here never change rounding-sensitive order: the compiler does not reassociate
// FP32 sums, and every product whose rounding error is needed is an explicit fmaf.
#pragma once

#include <cuda_runtime.h>
#include <string.h>

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

// x = hi + lo with hi = fl32(x) and lo = fl32(x - hi) (round to nearest even), ~2^-48 relative.
// For 2^-74 <= |x| < 2^127 the split is done on the bits of x with integer operations: this GPU
// runs FP64 arithmetic and conversions at a small fraction of its integer and FP32 rates.  The
// 53-bit significand M is rounded to 24 bits (q, ties to even), and x - hi = (M - q 2^29) 2^(E-52)
// is a signed integer of at most 29 bits times a power of two: its float conversion rounds as
// fl32(x - hi) does, and the power of two is added to the exponent field (no underflow in that
// range).  Zero is split on its bits as well; tiny and huge values take the FP64 conversions.
__host__ __device__ __forceinline__ void split_double(double x, float& hi, float& lo)
{
#ifdef __CUDA_ARCH__
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  memcpy(&b, &x, sizeof(b));
#endif
  const int E = (int)((b >> 52) & 0x7FF) - 1023;
  if ((b << 1) == 0ull) {  // +-0
    const unsigned int zb = (unsigned int)(b >> 32);
#ifdef __CUDA_ARCH__
    hi = __int_as_float((int)zb);
#else
    memcpy(&hi, &zb, sizeof(hi));
#endif
    lo = 0.f;
    return;
  }
  if (E >= -74 && E <= 126) {
    const unsigned long long M = (b & 0xFFFFFFFFFFFFFULL) | 0x10000000000000ULL;
    unsigned int q = (unsigned int)(M >> 29);  // [2^23, 2^24)
    const unsigned int r = (unsigned int)(M & 0x1FFFFFFFULL);
    const bool up = r > 0x10000000u || (r == 0x10000000u && (q & 1u));
    q += up ? 1u : 0u;  // 2^24 carries into the exponent below
    const unsigned int sgn = (unsigned int)(b >> 32) & 0x80000000u;
    const unsigned int hb = sgn | (((unsigned int)(E + 127) << 23) + (q - 0x800000u));
    const int d = (int)r - (up ? (1 << 29) : 0);
    unsigned int lb = 0u;
    if (d != 0) {
      const float fd = (float)d;  // round to nearest (|d| <= 2^28)
      unsigned int fb;
#ifdef __CUDA_ARCH__
      fb = (unsigned int)__float_as_int(fd);
#else
      memcpy(&fb, &fd, sizeof(fb));
#endif
      lb = (fb + ((unsigned int)(E - 52) << 23)) ^ sgn;
    }
#ifdef __CUDA_ARCH__
    hi = __int_as_float((int)hb);
    lo = __int_as_float((int)lb);
#else
    memcpy(&hi, &hb, sizeof(hi));
    memcpy(&lo, &lb, sizeof(lo));
#endif
    return;
  }
  hi = (float)x;
  lo = (float)(x - (double)hi);
}

__device__ __forceinline__ df df_from_double(double x)
{
  df r;
  split_double(x, r.hi, r.lo);
  return r;
}

// fl64(hi + lo) (round to nearest even), as (double)hi + (double)lo.  For normal hi and lo (or
// lo = 0) with lo's binade at least two below hi's (every renormalised or lazily formed
// double-float value) the sum is formed on integers: hi's significand
// widened to 53 bits plus 8 guard bits, lo's significand aligned to it (bits shifted out kept as
// a sticky bit), at most one normalising shift, then rounding on the guard bits.  Other values
// take the FP64 conversions.
__host__ __device__ __forceinline__ double df_to_double(df x)
{
  unsigned int hb, lb;
#ifdef __CUDA_ARCH__
  hb = (unsigned int)__float_as_int(x.hi);
  lb = (unsigned int)__float_as_int(x.lo);
#else
  memcpy(&hb, &x.hi, sizeof(hb));
  memcpy(&lb, &x.lo, sizeof(lb));
#endif
  const int eh = (int)((hb >> 23) & 0xFF), el = (int)((lb >> 23) & 0xFF);
  const bool lzero = (lb & 0x7FFFFFFFu) == 0u;
  if (eh >= 1 && eh <= 254 && (lzero || (el >= 1 && el <= eh - 2))) {
    const unsigned long long H = (unsigned long long)((hb & 0x7FFFFFu) | 0x800000u) << 37;  // 2^60 <= H < 2^61
    unsigned long long Lw = 0ull;
    if (!lzero) {
      const unsigned long long Ml = (unsigned long long)((lb & 0x7FFFFFu) | 0x800000u);
      const int g = eh - el;
      if (g <= 37)
        Lw = Ml << (37 - g);
      else if (g - 37 < 64)
        Lw = (Ml >> (g - 37)) | ((Ml & ((1ull << (g - 37)) - 1ull)) != 0ull ? 1ull : 0ull);
      else
        Lw = 1ull;  // sticky only
    }
    const bool same = ((hb ^ lb) & 0x80000000u) == 0u || lzero;
    unsigned long long S = same ? H + Lw : H - Lw;
    int E = eh - 127;
    if (S >> 61) {  // carry: one right shift, the bit shifted out joins the sticky bit
      S = (S >> 1) | (S & 1ull);
      ++E;
    } else if (!(S >> 60)) {  // borrow (H a power of two): one left shift
      S <<= 1;
      --E;
    }
    unsigned long long R = S >> 8;  // 53 bits, the leading one at bit 52
    const bool up = ((S >> 7) & 1ull) && ((S & 0x7Full) != 0ull || (R & 1ull));
    R += up ? 1ull : 0ull;
    if (R >> 53) {
      R >>= 1;
      ++E;
    }
    const unsigned long long bits = ((unsigned long long)(hb & 0x80000000u) << 32) |
                                    ((unsigned long long)(E + 1023) << 52) | (R & 0xFFFFFFFFFFFFFull);
    double d;
#ifdef __CUDA_ARCH__
    d = __longlong_as_double((long long)bits);
#else
    memcpy(&d, &bits, sizeof(d));
#endif
    return d;
  }
  return (double)x.hi + (double)x.lo;
}

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

// x * y without the final renormalisation: hi = fl(x.hi y.hi) and lo = its exact error plus
// the cross terms, |lo| <= ~2 ulp(hi) instead of ulp(hi)/2.  For a product that only feeds
// further double-float products or sums (which take hi and lo apart anyway).
__device__ __forceinline__ df df_mul_lazy(df x, df y)
{
  const float p = x.hi * y.hi;
  float e = fmaf(x.hi, y.hi, -p);
  e = fmaf(x.hi, y.lo, e);
  e = fmaf(x.lo, y.hi, e);
  return df_make(p, e);
}

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
