// Source construction of HSMA on the GPU (Sec. 2.3-2.4 of Fu & Gan, arXiv:1907.01724):
//   k_setup            (once per layout) per-system scalars eps, mu, R_tau, dy, gamma, sigma,
//                      dbar, the Kirkwood coefficients M_n (Sec. 2.2-2.3), recurrence tables
//                      and the Fibonacci points and weights of the auxiliary sphere (Sec. 2.4)
//   k_images_moments   trapezoid-modified Kelvin images q_K at r_K (Sec. 2.4) and the
//                      charge moments of the truncated correction coefficients
//   k_coef_reduce      correction coefficients hat A_nm (eq. phim), FP64
//   k_surface          Phi_corr and dPhi_corr/dr at the Fibonacci points and the monopole /
//                      dipole surface images (eqs. GreenSecond, approxG, threeintegrals,
//                      phicorrfinall)
// All arithmetic here is FP64; the FP32 path only stores its pair-sum records in FP32.
// FP64 division, square root and trigonometric functions are slow on this GPU, so everything
// that depends only on the parameters is done once in k_setup, and the per-step kernels use
// multiplications by stored reciprocals.
//
// Spherical harmonics are used as real, normalised solid harmonics
//   T^c_nm(x) = N_nm r^n P_n^m(cos t) cos(m f),  T^s_nm(x) = N_nm r^n P_n^m(cos t) sin(m f),
//   N_nm = sqrt((2 - delta_m0) (n-m)!/(n+m)!),
// so that the addition theorem reads sum_m [T^c(x)T^c(y) + T^s(x)T^s(y)] = r^n s^n P_n(cos angle).
// With x and y measured in units of a, eq. phim becomes
//   Phi_corr(y) = sum_nm A'_nm T_nm(y/a),
//   A'_nm = (k/(eps1 a)) sum_i q_i hat M'_{n,i} T_nm(x_i/a)
//         = (k/(eps1 a)) [ (M_n - gamma) U_nm - V_nm ],
//   U_nm = sum_i q_i T_nm(x_i/a),  V_nm = sum_i q_i c_i T_nm(x_i/a),
//   c_i = dbar (R_tau - r_K,i)/(2 r_K,i) = dbar (R_tau r_i/a^2 - 1)/2,
// which is the per-charge hat M'_{n,i} = M_n - gamma - c_i of Sec. 2.4 split into two
// charge moments.  Coefficient index: idx(n, m) = n^2 + n + m, m in [-n, n]; m < 0 holds
// the sine part of order |m|.
#include <math.h>

#include "df64.cuh"
#include "hsma_internal.cuh"

namespace hsma {

// ---------------------------------------------------------------------------------------
// Per-system scalars, tables and the quadrature grid.  Block s handles system s (thread 0:
// scalars and M_n; all threads: its Fibonacci points); block 0 also fills the tables.
// M_n uses the upward recurrence of the modified spherical Bessel functions: with
// t_n = mu k_{n-1}(mu)/k_n(mu) (k_{-1} = k_0), t_0 = mu and t_{n+1} = mu^2/(t_n + 2n + 1),
// mu k_n'/k_n = -(n+1) - t_n, i.e. S_n = -1/(n + 1 + t_n), and eq. Anuapp1 becomes
// M_n = -[(1 - eps)(n+1) + t_n] / [(1 + eps) n + 1 + t_n]  (finite at mu = 0).
// Fibonacci point j (Sec. 2.4): jj = j/2, z = -1 + 2 jj/F2, theta = arccos(z + sin(pi z)/pi),
// phi = pi jj F1/F2 (+ pi for odd j), weight w = (2 pi R_tau^2/F2)(1 + cos(pi z)).
__device__ __forceinline__ float2 pair_of(double x)
{
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}

__global__ void k_setup(SysDev* __restrict__ sys, int nsys, double* __restrict__ Mn, double* __restrict__ rec_a,
                        double* __restrict__ rec_b, double* __restrict__ sect, double* __restrict__ inv_np1,
                        float2* __restrict__ rec_a2, float2* __restrict__ rec_b2, float2* __restrict__ sect2,
                        int pmax, dbl4* __restrict__ surfx)
{
  if (blockIdx.x == 0) {
    const int ntri = (pmax + 1) * (pmax + 2) / 2;
    for (int t = threadIdx.x; t < ntri; t += blockDim.x) {
      int n = (int)floor((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while (n * (n + 1) / 2 > t) --n;
      while ((n + 1) * (n + 2) / 2 <= t) ++n;
      const int m = t - n * (n + 1) / 2;
      double A = 0.0, B = 0.0;
      if (n == m + 1) {
        A = sqrt(2.0 * m + 1.0);
      } else if (n >= m + 2) {
        A = (2.0 * n - 1.0) / sqrt((double)(n - m) * (double)(n + m));
        B = sqrt(((double)(n + m - 1) * (double)(n - m - 1)) / ((double)(n + m) * (double)(n - m)));
      }
      rec_a[t] = A;
      rec_b[t] = B;
      rec_a2[t] = pair_of(A);
      rec_b2[t] = pair_of(B);
    }
    for (int m = threadIdx.x; m <= pmax; m += blockDim.x) {
      sect[m] = (m >= 2) ? sqrt((2.0 * m - 1.0) / (2.0 * m)) : 1.0;
      sect2[m] = pair_of(sect[m]);
      inv_np1[m] = 1.0 / (m + 1.0);
    }
  }
  for (int s = blockIdx.x; s < nsys; s += gridDim.x) {
    SysDev& d = sys[s];
    if (threadIdx.x == 0) {
      d.eps = d.eps1 / d.eps2;
      d.mu = d.kappa * d.a;
      d.Rtau = (1.0 + d.tau) * d.a;
      d.dy = d.dy_rel * d.Rtau;
      d.gam = (d.eps - 1.0) / (d.eps + 1.0);
      d.sig = (1.0 + d.mu) / (1.0 + d.eps);
      d.dbar = d.gam * (1.0 - d.sig) - d.mu / (1.0 + d.eps);
      d.kc = d.coulk / d.eps1;
      d.inv_a = 1.0 / d.a;
      d.kc_a = d.kc / d.a;
      d.Rt_a = d.Rtau / d.a;
      d.inv_Rt = 1.0 / d.Rtau;
      double t = d.mu;
      for (int n = 0; n <= d.p; ++n) {
        Mn[d.mn + n] = -((1.0 - d.eps) * (n + 1) + t) / ((1.0 + d.eps) * n + 1.0 + t);
        t = d.mu * d.mu / (t + 2.0 * n + 1.0);
      }
    }
    const double Rt = (1.0 + d.tau) * d.a;
    for (int j = threadIdx.x; j < d.M; j += blockDim.x) {
      const int jj = j >> 1;
      const double z = -1.0 + 2.0 * (double)jj / (double)d.F2;
      double c = z + sin(kPi * z) / kPi;
      c = fmin(1.0, fmax(-1.0, c));
      const double theta = acos(c);
      const double phi = kPi * (double)jj * (double)d.F1 / (double)d.F2 + ((j & 1) ? kPi : 0.0);
      const double w = 2.0 * kPi * Rt * Rt / (double)d.F2 * (1.0 + cos(kPi * z));
      surfx[d.surf + j] = make_dbl4(Rt * sin(theta) * cos(phi), Rt * sin(theta) * sin(phi), Rt * cos(theta), w);
    }
  }
}

void launch_setup(SysDev* sys, int nsys, double* Mn, double* rec_a, double* rec_b, double* sect, double* inv_np1,
                  float2* rec_a2, float2* rec_b2, float2* sect2, int pmax, dbl4* surfx, cudaStream_t st)
{
  const int blocks = nsys < 4096 ? (nsys > 0 ? nsys : 1) : 4096;
  k_setup<<<blocks, 256, 0, st>>>(sys, nsys, Mn, rec_a, rec_b, sect, inv_np1, rec_a2, rec_b2, sect2, pmax, surfx);
}

// ---------------------------------------------------------------------------------------
// Arithmetic of the solid-harmonic steps: native FP64 for the FP64 path, double-float pairs
// (df64.cuh, ~2^-46 relative) on the FP32 pipes for the FP32 path.
template <class R>
struct Num;
template <>
struct Num<double> {
  static __device__ __forceinline__ double from(double x) { return x; }
  static __device__ __forceinline__ double from_int(int n) { return (double)n; }
  static __device__ __forceinline__ double to(double x) { return x; }
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double one() { return 1.0; }
  static __device__ __forceinline__ double ra(const Tables& t, int i) { return t.rec_a[i]; }
  static __device__ __forceinline__ double rb(const Tables& t, int i) { return t.rec_b[i]; }
  static __device__ __forceinline__ double sc(const Tables& t, int i) { return t.sect[i]; }
};
template <>
struct Num<df> {
  static __device__ __forceinline__ df from(double x) { return df_from_double(x); }
  static __device__ __forceinline__ df from_int(int n) { return df_make((float)n, 0.f); }
  static __device__ __forceinline__ double to(df x) { return df_to_double(x); }
  static __device__ __forceinline__ df zero() { return df_make(0.f, 0.f); }
  static __device__ __forceinline__ df one() { return df_make(1.f, 0.f); }
  static __device__ __forceinline__ df ra(const Tables& t, int i)
  {
    const float2 v = t.rec_a2[i];
    return df_make(v.x, v.y);
  }
  static __device__ __forceinline__ df rb(const Tables& t, int i)
  {
    const float2 v = t.rec_b2[i];
    return df_make(v.x, v.y);
  }
  static __device__ __forceinline__ df sc(const Tables& t, int i)
  {
    const float2 v = t.sect2[i];
    return df_make(v.x, v.y);
  }
};

// Real normalised solid harmonics of one point (u, v, w) (units of a), column m of the
// triangle, written to T[idx(n, +-m)] for n = m..p.  Sectoral: T_mm = s_m (u + i v) T_{m-1,m-1};
// vertical: T_{m+1,m} = sqrt(2m+1) w T_mm, T_nm = a_nm w T_{n-1,m} - b_nm rho^2 T_{n-2,m}.
template <class R>
__device__ __forceinline__ void solid_column(int m, int p, R u, R v, R w, R rho2, const Tables& tab,
                                             R* __restrict__ T)
{
  R cr = Num<R>::one(), ci = Num<R>::zero();
  for (int k = 1; k <= m; ++k) {
    const R f = Num<R>::sc(tab, k);
    const R nr = f * (cr * u - ci * v);
    const R ni = f * (cr * v + ci * u);
    cr = nr;
    ci = ni;
  }
  T[m * m + m + m] = cr;
  if (m) T[m * m + m - m] = ci;
  R pr = cr, pi = ci, qr = Num<R>::zero(), qi = Num<R>::zero();
  for (int n = m + 1; n <= p; ++n) {
    const int t = n * (n + 1) / 2 + m;
    const R A = Num<R>::ra(tab, t) * w, B = Num<R>::rb(tab, t) * rho2;
    const R nr = A * pr - B * qr;
    const R ni = A * pi - B * qi;
    T[n * n + n + m] = nr;
    if (m) T[n * n + n - m] = ni;
    qr = pr;
    qi = pi;
    pr = nr;
    pi = ni;
  }
}

// Split a double into an FP32 high part and the FP32-rounded residual (x ~ hi + lo).
__device__ __forceinline__ void split2(double x, float& hi, float& lo)
{
  hi = __double2float_rn(x);
  lo = __double2float_rn(x - (double)hi);
}

constexpr int kMomThreads = 256;  // moment blocks hold up to kMomTile charges
constexpr int kMomWarps = kMomThreads / 32;

// Kelvin images (Sec. 2.4): r_K = a^2/r along xhat, q_K = (q/a)[gamma r_K + dbar (R_tau - r_K)/2].
// Records: real charge (x, k q/eps1) and Kelvin image (r_K xhat, k q_K/eps1); FP32 path stores
// (hi x, hi y, hi z, Q) and (lo x, lo y, lo z, 0).
template <int MAXJ, class R>
__global__ __launch_bounds__(kMomThreads) void k_images_moments(
    const SysDev* __restrict__ sys, const int2* __restrict__ items, const double* __restrict__ xyz,
    const double* __restrict__ q, Tables tab, float4* __restrict__ src_hi, float4* __restrict__ src_lo,
    dbl4* __restrict__ src64, int prec, double* __restrict__ mom, int mom_stride, int G, int* __restrict__ status)
{
  extern __shared__ double sm[];
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int n = S.n, P = S.P, p = S.p;
  const double a = S.a, kc = S.kc, gam = S.gam, dbar = S.dbar, Rtau = S.Rtau, inv_a = S.inv_a;
  const int c0 = it.y * S.mom_tile;
  const int c1 = min(n, c0 + S.mom_tile);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  static_assert(sizeof(R) == sizeof(double), "moment arithmetic uses 8-byte values");
  R* T = reinterpret_cast<R*>(sm);                 // [G][P]
  R* qv = T + (size_t)G * P;                       // [G]
  R* qc = qv + G;                                  // [G]
  double* red = reinterpret_cast<double*>(qc + G);  // [kMomWarps]

  // images
  double r0 = 0.0;
  for (int i = c0 + tid; i < c1; i += kMomThreads) {
    const long long gi = S.chg + i;
    const double x = xyz[3 * gi], y = xyz[3 * gi + 1], z = xyz[3 * gi + 2], qi = q[gi];
    // r, r_K and the Kelvin point use separately rounded IEEE operations (no FMA contraction):
    // a charge at distance d from the interface sits ~2d from its own image, so one ulp in r
    // would be amplified by r/d in the image term
    const double r = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
    if (!(r < a) || !isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(qi)) atomicOr(status, kStOutside);
    double kx, ky, kz, QK;
    if (r <= kCentreRel * a) {
      // image at infinity: constant potential k q/(eps1 a) (gamma - dbar/2) at every target
      r0 += S.kc_a * qi * (gam - 0.5 * dbar);
      kx = 1e15 * a;
      ky = 0.0;
      kz = 0.0;
      QK = 0.0;
    } else {
      const double ar = __ddiv_rn(a, r);
      const double s = __dmul_rn(ar, ar);
      const double rK = __dmul_rn(ar, a);
      kx = __dmul_rn(s, x);
      ky = __dmul_rn(s, y);
      kz = __dmul_rn(s, z);
      QK = kc * (qi * inv_a * (gam * rK + dbar * (Rtau - rK) * 0.5));
    }
    const long long sr = S.src + i, sk = S.src + n + i;
    if (prec == HSMA_FP64) {
      src64[sr] = make_dbl4(x, y, z, kc * qi);
      src64[sk] = make_dbl4(kx, ky, kz, QK);
    } else {
      float hx, hy, hz, lx, ly, lz;
      split2(x, hx, lx);
      split2(y, hy, ly);
      split2(z, hz, lz);
      src_hi[sr] = make_float4(hx, hy, hz, (float)(kc * qi));
      src_lo[sr] = make_float4(lx, ly, lz, 0.f);
      split2(kx, hx, lx);
      split2(ky, hy, ly);
      split2(kz, hz, lz);
      src_hi[sk] = make_float4(hx, hy, hz, (float)QK);
      src_lo[sk] = make_float4(lx, ly, lz, 0.f);
    }
  }
  // block sum of the centre-charge constants (fixed order)
  for (int o = 16; o > 0; o >>= 1) r0 += __shfl_xor_sync(0xffffffffu, r0, o);
  if (lane == 0) red[warp] = r0;
  __syncthreads();
  double* out = mom + (size_t)(S.mom + it.y) * mom_stride;
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kMomWarps; ++w) s += red[w];
    out[2 * P] = s;
  }

  // charge moments U_nm, V_nm
  R accU[MAXJ], accV[MAXJ];
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) accU[j] = accV[j] = Num<R>::zero();
  for (int g0 = c0; g0 < c1; g0 += G) {
    const int gcount = min(G, c1 - g0);
    if (warp < gcount) {
      const long long gi = S.chg + g0 + warp;
      const double x = xyz[3 * gi] * inv_a, y = xyz[3 * gi + 1] * inv_a, z = xyz[3 * gi + 2] * inv_a;
      const double rho2 = x * x + y * y + z * z;
      R* Tg = T + (size_t)warp * P;
      const R xr = Num<R>::from(x), yr = Num<R>::from(y), zr = Num<R>::from(z), r2r = Num<R>::from(rho2);
      for (int m = lane; m <= p; m += 32) solid_column<R>(m, p, xr, yr, zr, r2r, tab, Tg);
      if (lane == 0) {
        const double qi = q[gi];
        qv[warp] = Num<R>::from(qi);
        qc[warp] = Num<R>::from(qi * (dbar * (S.Rt_a * sqrt(rho2) - 1.0) * 0.5));
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
      const int idx = tid + j * kMomThreads;
      if (idx < P) {
        R u = accU[j], v = accV[j];
        for (int g = 0; g < gcount; ++g) {
          const R t = T[(size_t)g * P + idx];
          u = qv[g] * t + u;
          v = qc[g] * t + v;
        }
        accU[j] = u;
        accV[j] = v;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) {
    const int idx = tid + j * kMomThreads;
    if (idx < P) {
      out[idx] = Num<R>::to(accU[j]);
      out[P + idx] = Num<R>::to(accV[j]);
    }
  }
}

int moment_smem_group(int maxP)
{
  const size_t budget = 160 * 1024;
  int G = (int)(budget / ((size_t)maxP * 8 + 16));
  if (G > kMomWarps) G = kMomWarps;
  if (G < 1) G = 1;
  return G;
}

template <int MAXJ>
static void launch_im(const SysDev* sys, const int2* items, int nitems, int maxP, const double* xyz, const double* q,
                      Tables tab, float4* src_hi, float4* src_lo, dbl4* src64, int prec, double* mom,
                      int mom_stride, int* status, cudaStream_t st)
{
  const int G = moment_smem_group(maxP);
  const size_t smem = ((size_t)G * maxP + 2 * G + kMomWarps) * sizeof(double);
  if (prec == HSMA_FP64)
    k_images_moments<MAXJ, double><<<nitems, kMomThreads, smem, st>>>(sys, items, xyz, q, tab, src_hi, src_lo, src64,
                                                                       prec, mom, mom_stride, G, status);
  else
    k_images_moments<MAXJ, df><<<nitems, kMomThreads, smem, st>>>(sys, items, xyz, q, tab, src_hi, src_lo, src64,
                                                                   prec, mom, mom_stride, G, status);
}

void launch_images_moments(const SysDev* sys, const int2* items, int nitems, int maxP, const double* xyz,
                           const double* q, Tables tab, float4* src_hi, float4* src_lo, dbl4* src64, int prec,
                           double* mom, int mom_stride, int* status, cudaStream_t st)
{
  if (nitems <= 0) return;
  const int J = (maxP + kMomThreads - 1) / kMomThreads;
  if (J <= 1)
    launch_im<1>(sys, items, nitems, maxP, xyz, q, tab, src_hi, src_lo, src64, prec, mom, mom_stride, status, st);
  else if (J <= 2)
    launch_im<2>(sys, items, nitems, maxP, xyz, q, tab, src_hi, src_lo, src64, prec, mom, mom_stride, status, st);
  else if (J <= 4)
    launch_im<4>(sys, items, nitems, maxP, xyz, q, tab, src_hi, src_lo, src64, prec, mom, mom_stride, status, st);
  else if (J <= 8)
    launch_im<8>(sys, items, nitems, maxP, xyz, q, tab, src_hi, src_lo, src64, prec, mom, mom_stride, status, st);
  else if (J <= 16)
    launch_im<16>(sys, items, nitems, maxP, xyz, q, tab, src_hi, src_lo, src64, prec, mom, mom_stride, status, st);
  else
    launch_im<26>(sys, items, nitems, maxP, xyz, q, tab, src_hi, src_lo, src64, prec, mom, mom_stride, status, st);
}

// ---------------------------------------------------------------------------------------
// hat A'_nm = (k/(eps1 a)) [(M_n - gamma) U_nm - V_nm].  A block owns kCoefChunk coefficients
// (one per lane); its kCoefWarps warps split the moment blocks (warp w takes blocks w,
// w + kCoefWarps, ...), and warp 0 adds the warp sums in order, so the result does not depend
// on scheduling.
constexpr int kCoefWarps = 32;
__global__ __launch_bounds__(kCoefWarps * 32) void k_coef_reduce(const SysDev* __restrict__ sys,
                                                                 const int2* __restrict__ items,
                                                                 const double* __restrict__ mom, int mom_stride,
                                                                 const double* __restrict__ Mn,
                                                                 double* __restrict__ coef, double* __restrict__ r0)
{
  __shared__ double su[kCoefWarps][kCoefChunk], sv[kCoefWarps][kCoefChunk], sr[kCoefWarps];
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int P = S.P;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int idx = it.y * kCoefChunk + lane;
  const double* base = mom + (size_t)S.mom * mom_stride;
  double U = 0.0, V = 0.0, R = 0.0;
  if (idx < P)
    for (int b = warp; b < S.mom_blocks; b += kCoefWarps) {
      U += base[(size_t)b * mom_stride + idx];
      V += base[(size_t)b * mom_stride + P + idx];
    }
  if (it.y == 0 && lane == 0)
    for (int b = warp; b < S.mom_blocks; b += kCoefWarps) R += base[(size_t)b * mom_stride + 2 * P];
  su[warp][lane] = U;
  sv[warp][lane] = V;
  if (lane == 0) sr[warp] = R;
  __syncthreads();
  if (warp == 0) {
    U = 0.0;
    V = 0.0;
    for (int w = 0; w < kCoefWarps; ++w) {
      U += su[w][lane];
      V += sv[w][lane];
    }
    if (idx < P) {
      int nn = (int)sqrtf((float)idx);
      while (nn * nn > idx) --nn;
      while ((nn + 1) * (nn + 1) <= idx) ++nn;
      coef[S.coef + idx] = S.kc_a * ((Mn[S.mn + nn] - S.gam) * U - V);
    }
    if (it.y == 0 && lane == 0) {
      double s = 0.0;
      for (int w = 0; w < kCoefWarps; ++w) s += sr[w];
      r0[it.x] = s;
    }
  }
}

void launch_coef_reduce(const SysDev* sys, const int2* items, int nitems, const double* mom, int mom_stride,
                        const double* Mn, double* coef, double* r0, cudaStream_t st)
{
  if (nitems <= 0) return;
  k_coef_reduce<<<nitems, kCoefWarps * 32, 0, st>>>(sys, items, mom, mom_stride, Mn, coef, r0);
}

// ---------------------------------------------------------------------------------------
// Surface images.  One warp per Fibonacci point y (from k_setup); lane m sums column m of
//   Phi = sum A'_nm T_nm(y/a),   dPhi/dr = sum n A'_nm T_nm(y/a) / R_tau,
// then a fixed-order shuffle reduction.  Records (Green's second identity + central
// difference, eq. threeintegrals): monopole Q0 = w dPhi/dr / (4 pi) at y = R_tau yhat and
// dipole D = w Phi / (4 pi) between y_- and y_+.
constexpr int kSurfThreads = 256;
constexpr int kSurfWarps = kSurfThreads / 32;
static_assert(kSurfWarps == kSurfPointsPerBlock, "one warp per surface point");

template <class R>
__global__ __launch_bounds__(kSurfThreads) void k_surface(const SysDev* __restrict__ sys,
                                                          const int2* __restrict__ items,
                                                          const double* __restrict__ coef, Tables tab,
                                                          float4* __restrict__ surf_a, float4* __restrict__ surf_b,
                                                          dbl4* __restrict__ surf64_a,
                                                          double* __restrict__ surf64_b,
                                                          const dbl4* __restrict__ surfx,
                                                          double2* __restrict__ surfqd, int prec)
{
  extern __shared__ double sm[];
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int P = S.P, p = S.p, M = S.M;
  R* A = reinterpret_cast<R*>(sm);  // [P]
  for (int i = threadIdx.x; i < P; i += kSurfThreads) A[i] = Num<R>::from(coef[S.coef + i]);
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = it.y * kSurfWarps + warp;
  if (j >= M) return;
  const long long o = S.surf + j;
  const dbl4 yw = surfx[o];
  const double ud = yw.x * S.inv_a, vd = yw.y * S.inv_a, wd = yw.z * S.inv_a;
  const R u = Num<R>::from(ud), v = Num<R>::from(vd), ww = Num<R>::from(wd);
  const R rho2 = Num<R>::from(ud * ud + vd * vd + wd * wd);
  R phr = Num<R>::zero(), dphr = Num<R>::zero();
  for (int m = lane; m <= p; m += 32) {
    R cr = Num<R>::one(), ci = Num<R>::zero();
    for (int k = 1; k <= m; ++k) {
      const R f = Num<R>::sc(tab, k);
      const R nr = f * (cr * u - ci * v);
      const R ni = f * (cr * v + ci * u);
      cr = nr;
      ci = ni;
    }
    R t = m ? A[m * m + m + m] * cr + A[m * m + m - m] * ci : A[0] * cr;
    phr = phr + t;
    dphr = Num<R>::from_int(m) * t + dphr;
    R pr = cr, pi = ci, qr = Num<R>::zero(), qi = Num<R>::zero();
    for (int n = m + 1; n <= p; ++n) {
      const int tt = n * (n + 1) / 2 + m;
      const R Aa = Num<R>::ra(tab, tt) * ww, Bb = Num<R>::rb(tab, tt) * rho2;
      const R nr = Aa * pr - Bb * qr;
      const R ni = Aa * pi - Bb * qi;
      t = m ? A[n * n + n + m] * nr + A[n * n + n - m] * ni : A[n * n + n] * nr;
      phr = phr + t;
      dphr = Num<R>::from_int(n) * t + dphr;
      qr = pr;
      qi = pi;
      pr = nr;
      pi = ni;
    }
  }
  double ph = Num<R>::to(phr), dph = Num<R>::to(dphr);
  for (int off = 16; off > 0; off >>= 1) {
    ph += __shfl_xor_sync(0xffffffffu, ph, off);
    dph += __shfl_xor_sync(0xffffffffu, dph, off);
  }
  if (lane == 0) {
    const double w4 = yw.w * (0.25 / kPi);
    const double Q0 = w4 * (dph * S.inv_Rt);
    const double D = w4 * ph;
    surfqd[o] = make_double2(Q0, D);
    if (prec == HSMA_FP64) {
      surf64_a[o] = make_dbl4(yw.x, yw.y, yw.z, Q0);
      surf64_b[o] = D;
    } else {
      // FP32 path: the dipole is applied through its Delta y -> 0 limit
      // D (R_tau - x.yhat)/d^3 = Dp ((x - y).y) / d^3 with Dp = -D/R_tau
      surf_a[o] = make_float4((float)yw.x, (float)yw.y, (float)yw.z, (float)Q0);
      surf_b[o] = make_float4((float)(-D * S.inv_Rt), 0.f, 0.f, 0.f);
    }
  }
}

void launch_surface(const SysDev* sys, const int2* items, int nitems, int maxP, const double* coef, Tables tab,
                    float4* surf_a, float4* surf_b, dbl4* surf64_a, double* surf64_b, dbl4* surfx, double2* surfqd,
                    int prec, cudaStream_t st)
{
  if (nitems <= 0) return;
  const size_t smem = (size_t)maxP * sizeof(double);
  if (prec == HSMA_FP64)
    k_surface<double><<<nitems, kSurfThreads, smem, st>>>(sys, items, coef, tab, surf_a, surf_b, surf64_a, surf64_b,
                                                          surfx, surfqd, prec);
  else
    k_surface<df><<<nitems, kSurfThreads, smem, st>>>(sys, items, coef, tab, surf_a, surf_b, surf64_a, surf64_b,
                                                      surfx, surfqd, prec);
}

template <class R>
static void moment_attrs()
{
  cudaFuncSetAttribute(k_images_moments<1, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_images_moments<2, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_images_moments<4, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_images_moments<8, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_images_moments<16, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_images_moments<26, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_surface<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
}

void init_source_kernels()
{
  moment_attrs<double>();
  moment_attrs<df>();
}

}  // namespace hsma
