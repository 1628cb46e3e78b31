// Source construction of HSMA on the GPU (Sec. 2.3-2.4 of Fu & Gan, arXiv:1907.01724):
//   k_setup            (once per layout) per-system scalars eps, mu, R_tau, dy, gamma, sigma,
//                      dbar, the Kirkwood coefficients M_n (Sec. 2.2-2.3), recurrence tables
//                      and the Fibonacci points and weights of the auxiliary sphere (Sec. 2.4)
//   k_surface_basis    (once per layout) solid harmonics of the auxiliary-sphere points
//   k_images           trapezoid-modified Kelvin images q_K at r_K (Sec. 2.4) and the pair-sum
//                      records, in spatial order, with the bounding box of every 32 records
//   k_moment_prep,     charge moments of the truncated correction coefficients: FP32 path (a
//   k_moment_units     warp per 32 charges and column pair, double-float)
//   k_moments          the same on the FP64 path (a block per tile of charges, FP64)
//   k_coef_reduce      correction coefficients hat A_nm (eq. phim)
//   k_surface_mat      Phi_corr and dPhi_corr/dr at the Fibonacci points and the monopole /
//                      dipole surface images (eqs. GreenSecond, approxG, threeintegrals,
//                      phicorrfinall)
// Geometry (images, radii, centre constants) is FP64.  The solid-harmonic sums run in FP64 on
// the FP64 path and in double-float arithmetic (df64.cuh) on the FP32 path: FP64 on this GPU
// runs at about 1/73 of the FP32 rate, and so do its division, square root and trigonometric
// functions, so everything that depends only on the parameters is done once per layout, and
// the per-step kernels keep FP64 to a few operations per charge.
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
// which is the per-charge hat M'_{n,i} = M_n - gamma - c_i of Sec. 2.4; the moment kernel forms
// the weights q_i hat M'_{n,i} once per (n, charge) and accumulates one sum per coefficient.
// Coefficient index: idx(n, m) = n^2 + n + m, m in [-n, n]; m < 0 holds the sine part of order
// |m|.
#include <math.h>

#include <algorithm>
#include <cmath>

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
  float2 r;
  split_double(x, r.x, r.y);
  return r;
}

// Vertical recurrence coefficients of the normalised solid harmonics below the diagonal:
// T_nm = a_nm w T_{n-1,m} - b_nm rho^2 T_{n-2,m} (a_{m+1,m} = sqrt(2m+1), b_{m+1,m} = 0).
__device__ __forceinline__ void rec_coef(int n, int m, double& A, double& B)
{
  A = 0.0;
  B = 0.0;
  if (n == m + 1) {
    A = sqrt(2.0 * m + 1.0);
  } else if (n >= m + 2) {
    A = (2.0 * n - 1.0) / sqrt((double)(n - m) * (double)(n + m));
    B = sqrt(((double)(n + m - 1) * (double)(n - m - 1)) / ((double)(n + m) * (double)(n - m)));
  }
}

__global__ void k_setup(SysDev* __restrict__ sys, int nsys, double* __restrict__ Mn, double* __restrict__ rec_a,
                        double* __restrict__ rec_b, double* __restrict__ sect, double* __restrict__ inv_np1,
                        float2* __restrict__ rec_a2, float2* __restrict__ rec_b2, float2* __restrict__ sect2,
                        float2* __restrict__ mtab, int pmax, dbl4* __restrict__ surfx)
{
  if (blockIdx.x == 0) {
    const int ntri = (pmax + 1) * (pmax + 2) / 2;
    for (int t = threadIdx.x; t < ntri; t += blockDim.x) {
      int n = (int)floor((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
      while (n * (n + 1) / 2 > t) --n;
      while ((n + 1) * (n + 2) / 2 <= t) ++n;
      const int m = t - n * (n + 1) / 2;
      double A, B;
      rec_coef(n, m, A, B);
      rec_a[t] = A;
      rec_b[t] = B;
      rec_a2[t] = pair_of(A);
      rec_b2[t] = pair_of(B);
    }
    // the rescaled column chain of k_moment_units, one column per thread: with
    // e_nm = prod_{k=m+1..n} a_km / 2, S_n = T_nm / (e_nm sprod_m z^m) obeys
    // S_n = 2 w S_{n-1} - beta_nm rho^2 S_{n-2}, beta_nm = 4 b_nm / (a_nm a_{n-1,m}), S_m = 1
    // (no table factor left in the chain)
    // (beta rows past pmax, up to pmax + kMomUnitSteps, only feed chain steps whose values are
    // discarded)
    const int nbeta = moment_beta_slots(pmax);
    for (int m = threadIdx.x; m <= pmax; m += blockDim.x) {
      double sp = 1.0;
      for (int k = 2; k <= m; ++k) sp *= sqrt((2.0 * k - 1.0) / (2.0 * k));
      double e = 1.0, Aprev = 0.0;
      for (int n = m; n <= pmax + kMomUnitSteps; ++n) {
        double A, B;
        rec_coef(n, m, A, B);
        if (n > m) e *= 0.5 * A;
        const int t = n * (n + 1) / 2 + m;
        mtab[t] = pair_of(n >= m + 2 ? 4.0 * B / (A * Aprev) : 0.0);
        if (n <= pmax) mtab[nbeta + t] = pair_of(e * sp);
        Aprev = A;
      }
    }
    for (int m = threadIdx.x; m <= pmax; m += blockDim.x) {
      sect[m] = (m >= 2) ? sqrt((2.0 * m - 1.0) / (2.0 * m)) : 1.0;
      sect2[m] = pair_of(sect[m]);
      inv_np1[m] = 1.0 / (m + 1.0);
      sect2[pmax + 1 + m] = pair_of((2.0 * m + 1.0) / (m + 1.0));  // Legendre: P_{n+1} = a P_n t - b P_{n-1}
      sect2[2 * (pmax + 1) + m] = pair_of((double)m / (m + 1.0));
      double sp = 1.0;
      for (int k = 2; k <= m; ++k) sp *= sqrt((2.0 * k - 1.0) / (2.0 * k));
      sect[pmax + 1 + m] = sp;
      sect2[3 * (pmax + 1) + m] = pair_of(sp);
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
      d.f_kc = pair_of(d.kc);
      d.f_a = pair_of(d.a);
      d.f_a2 = pair_of(d.a * d.a);
      d.f_qk1 = pair_of(d.kc_a * (d.gam - 0.5 * d.dbar));
      d.f_qk0 = pair_of(d.kc_a * d.dbar * d.Rtau * 0.5);
      d.f_rc2 = (float)(4.0 * (kCentreRel * d.a) * (kCentreRel * d.a));
      d.f_inv_a = pair_of(d.inv_a);
      d.f_hdbar = pair_of(0.5 * d.dbar);
      d.f_Rt_a = pair_of(d.Rt_a);
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
                  float2* rec_a2, float2* rec_b2, float2* sect2, float2* mtab, int pmax, dbl4* surfx, cudaStream_t st)
{
  const int blocks = nsys < 4096 ? (nsys > 0 ? nsys : 1) : 4096;
  k_setup<<<blocks, 256, 0, st>>>(sys, nsys, Mn, rec_a, rec_b, sect, inv_np1, rec_a2, rec_b2, sect2, mtab, pmax,
                                  surfx);
}

// ---------------------------------------------------------------------------------------
// Arithmetic of the solid-harmonic steps: native FP64 for the FP64 path, double-float pairs
// (df64.cuh, ~2^-46 relative) on the FP32 pipes for the FP32 path.
template <class R>
struct Num;
template <>
struct Num<double> {
  static constexpr bool is_df = false;
  static __device__ __forceinline__ double from(double x) { return x; }
  static __device__ __forceinline__ double from_df(df x) { return df_to_double(x); }
  static __device__ __forceinline__ double from_int(int n) { return (double)n; }
  static __device__ __forceinline__ double to(double x) { return x; }
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double one() { return 1.0; }
  static __device__ __forceinline__ double ra(const Tables& t, int i) { return t.rec_a[i]; }
  static __device__ __forceinline__ double rb(const Tables& t, int i) { return t.rec_b[i]; }
  static __device__ __forceinline__ double sc(const Tables& t, int i) { return t.sect[i]; }
  // a value in an 8-byte slot of a double-typed buffer
  static __device__ __forceinline__ double ld(const double* p, long long i) { return p[i]; }
  static __device__ __forceinline__ void st(double* p, long long i, double v) { p[i] = v; }
  static __device__ __forceinline__ double shfl(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
  static __device__ __forceinline__ double coefv(const double* c, const float2*, long long i) { return c[i]; }
  static __device__ __forceinline__ double mul_sub(double a, double x, double b, double y) { return a * x - b * y; }
  static __device__ __forceinline__ double acc(double s, double a, double b) { return a * b + s; }
  static __device__ __forceinline__ double norm(double x) { return x; }
};
template <>
struct Num<df> {
  static constexpr bool is_df = true;
  static __device__ __forceinline__ df from(double x) { return df_from_double(x); }
  static __device__ __forceinline__ df from_df(df x) { return x; }
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
  // a (hi, lo) pair in an 8-byte slot of a double-typed buffer
  static __device__ __forceinline__ df ld(const double* p, long long i)
  {
    const float2 v = reinterpret_cast<const float2*>(p)[i];
    return df_make(v.x, v.y);
  }
  static __device__ __forceinline__ void st(double* p, long long i, df v)
  {
    reinterpret_cast<float2*>(p)[i] = make_float2(v.hi, v.lo);
  }
  static __device__ __forceinline__ df shfl(df v, int o)
  {
    return df_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
  }
  static __device__ __forceinline__ df coefv(const double*, const float2* c2, long long i)
  {
    const float2 v = c2[i];
    return df_make(v.x, v.y);
  }
  static __device__ __forceinline__ df mul_sub(df a, df x, df b, df y) { return df_mul_sub(a, x, b, y); }
  static __device__ __forceinline__ df acc(df s, df a, df b) { return df_acc(s, a, b); }
  static __device__ __forceinline__ df norm(df x) { return df_norm(x); }
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
    const R nr = f * Num<R>::mul_sub(cr, u, ci, v);
    const R ni = f * Num<R>::mul_sub(cr, v, -ci, u);
    cr = nr;
    ci = ni;
  }
  T[m * m + m + m] = cr;
  if (m) T[m * m + m - m] = ci;
  R pr = cr, pi = ci, qr = Num<R>::zero(), qi = Num<R>::zero();
  for (int n = m + 1; n <= p; ++n) {
    const int t = n * (n + 1) / 2 + m;
    const R A = Num<R>::ra(tab, t) * w, B = Num<R>::rb(tab, t) * rho2;
    const R nr = Num<R>::mul_sub(A, pr, B, qr);
    const R ni = Num<R>::mul_sub(A, pi, B, qi);
    T[n * n + n + m] = nr;
    if (m) T[n * n + n - m] = ni;
    qr = pr;
    qi = pi;
    pr = nr;
    pi = ni;
  }
}

// The columns m1 = j and m2 = p - j (j <= p/2) of one point, for the moment kernel: one thread
// per column pair keeps every lane of a warp busy for about 2p steps (one thread per column
// leaves the warp waiting for its longest sectoral and vertical chains).  The sectoral
// values are T_mm = sprod_m (u + i v)^m, with the power carried from m1 to m2; below the
// diagonal the vertical recurrence is real, T_nm = Q_n T_mm with Q_m = 1, Q_{m-1} = 0,
// Q_n = a_nm w Q_{n-1} - b_nm rho^2 Q_{n-2}.  ra, rb, sp: a_nm, b_nm (index n(n+1)/2 + m)
// and sprod in the arithmetic R.
template <class R>
__device__ __forceinline__ void solid_vertical(int m, int p, R w, R rho2, R cr, R ci, const R* __restrict__ ra,
                                               const R* __restrict__ rb, R* __restrict__ T)
{
  T[m * m + 2 * m] = cr;
  if (m) T[m * m] = ci;
  R q1 = Num<R>::one(), q2 = Num<R>::zero();
  int t = (m + 1) * (m + 2) / 2 + m;  // table index of (n, m), n = m + 1
  int i0 = (m + 1) * (m + 2);         // coefficient index of (n, 0)
  for (int n = m + 1; n <= p; ++n) {
    const R A = ra[t] * w, B = rb[t] * rho2;
    const R qn = Num<R>::mul_sub(A, q1, B, q2);
    T[i0 + m] = qn * cr;
    if (m) T[i0 - m] = qn * ci;
    q2 = q1;
    q1 = qn;
    t += n + 1;
    i0 += 2 * n + 2;
  }
}

template <class R>
__device__ __forceinline__ void solid_pair(int j, int p, R u, R v, R w, R rho2, const R* __restrict__ ra,
                                           const R* __restrict__ rb, const R* __restrict__ sp, R* __restrict__ T)
{
  const int m1 = j, m2 = p - j;
  R zr = Num<R>::one(), zi = Num<R>::zero();
  R c1r = Num<R>::one(), c1i = Num<R>::zero();
  for (int k = 1; k <= m2; ++k) {
    const R nr = Num<R>::mul_sub(zr, u, zi, v);
    const R ni = Num<R>::mul_sub(zr, v, -zi, u);
    zr = nr;
    zi = ni;
    if (k == m1) {
      c1r = sp[m1] * zr;
      c1i = sp[m1] * zi;
    }
  }
  solid_vertical<R>(m1, p, w, rho2, c1r, c1i, ra, rb, T);
  if (m2 != m1) solid_vertical<R>(m2, p, w, rho2, sp[m2] * zr, sp[m2] * zi, ra, rb, T);
}



constexpr int kMomThreads = 352;  // a moment block holds at most kMomTile <= kMomThreads charges
constexpr int kMomWarps = kMomThreads / 32;
// Slots of the recurrence tables (a_nm, b_nm over the triangle n <= pmax, and the sectoral
// factors) that k_moments keeps in shared memory when they take at most kMomTableSlots slots.
constexpr size_t kMomTableSlots = 4096;
static_assert(kMomTile <= kMomThreads, "one charge per thread in the preparation pass");
static_assert(kOrderBlock % 64 == 0, "k_images splits an order item into 64-thread blocks");

// Kelvin image of one charge (Sec. 2.4): r_K = a^2/r along xhat,
// q_K = (q/a)[gamma r_K + dbar (R_tau - r_K)/2], strength k q_K/eps1.  r, r_K and the image
// point use separately rounded IEEE operations (no FMA contraction): a charge at distance d from
// the interface sits ~2d from its own image, so one ulp in r would be amplified by r/d in the
// image term.  A charge within kCentreRel a of the centre has its image at infinity: a constant
// potential k q/(eps1 a) (gamma - dbar/2) at every target (returned in C; the record then has
// zero strength).
struct KelvinRec {
  double r, kx, ky, kz, QK, C;
};
__device__ __forceinline__ KelvinRec kelvin_rec(const SysDev& S, double x, double y, double z, double qi)
{
  KelvinRec k;
  k.r = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
  k.C = 0.0;
  if (k.r <= kCentreRel * S.a) {
    k.C = S.kc_a * qi * (S.gam - 0.5 * S.dbar);
    k.kx = 1e15 * S.a;
    k.ky = 0.0;
    k.kz = 0.0;
    k.QK = 0.0;
  } else {
    const double ar = __ddiv_rn(S.a, k.r);
    const double s = __dmul_rn(ar, ar);
    const double rK = __dmul_rn(ar, S.a);
    k.kx = __dmul_rn(s, x);
    k.ky = __dmul_rn(s, y);
    k.kz = __dmul_rn(s, z);
    k.QK = S.kc * (qi * S.inv_a * (S.gam * rK + S.dbar * (S.Rtau - rK) * 0.5));
  }
  return k;
}

// Pair-sum records in the spatial order of k_order.cu: item (s, b) covers sorted positions
// [kOrderBlock b, kOrderBlock (b + 1)); sorted position i holds input charge perm[i].  Real
// record (x, k q/eps1) at src + i and Kelvin record at src + n + i; the FP32 path stores
// (hi x, hi y, hi z, Q) and (lo x, lo y, lo z, 0) and, per warp (32 consecutive records), the
// bounding box of the hi coordinates (min, max as two float4) of the real and of the Kelvin
// records.
// Blocks of 64 threads (four per item): small blocks find room beside the moment kernel; the
// FP64 path's image geometry is FP64, which this GPU issues at a low rate per SM, so it is
// spread over four times as many SMs.
constexpr int kImgThreads = 64;
constexpr int kImgSplit = kOrderBlock / kImgThreads;
__global__ __launch_bounds__(kImgThreads) void k_images(const SysDev* __restrict__ sys, const int2* __restrict__ items,
                                                        const double* __restrict__ xyz, const double* __restrict__ q,
                                                        const float4* __restrict__ xs, const int* __restrict__ perm,
                                                        int* __restrict__ iperm,
                                                        float4* __restrict__ src_hi, float4* __restrict__ src_lo,
                                                        dbl4* __restrict__ src64, float4* __restrict__ boxes, int prec,
                                                        int* __restrict__ status)
{
  // the item and the system's constants are loaded while k_order_sort runs (this kernel is
  // its programmatic dependent; a copy, so the loads precede the wait), perm after it
  const int2 it = items[blockIdx.x / kImgSplit];
  const SysDev S = sys[it.x];
  const int n = S.n;
  const int i = it.y * kOrderBlock + (blockIdx.x % kImgSplit) * kImgThreads + threadIdx.x;
  const int lane = threadIdx.x & 31;
  grid_dependency_wait();
  float bmin[6], bmax[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    bmin[d] = 3.0e38f;
    bmax[d] = -3.0e38f;
  }
  if (prec == HSMA_FP64) {
    if (i < n) {
      const long long gi = S.chg + perm[S.chg + i];
      iperm[gi] = i;
      const double x = xyz[3 * gi], y = xyz[3 * gi + 1], z = xyz[3 * gi + 2], qi = q[gi];
      const KelvinRec k = kelvin_rec(S, x, y, z, qi);
      if (!(k.r < S.a) || !isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(qi)) atomicOr(status, kStOutside);
      src64[S.src + i] = make_dbl4(x, y, z, S.kc * qi);
      src64[S.src + n + i] = make_dbl4(k.kx, k.ky, k.kz, k.QK);
    }
  } else {
    // from the (hi, lo) split of k_order_keys, in double-float arithmetic on the FP32 pipes
    // (FP64 only for a charge within 2 kCentreRel a of the centre): r^2, s = a^2 / r^2, the
    // Kelvin point s x (its (hi, lo) pair is the record's split), r_K = a sqrt(s) and
    // q_K = q (qk1 r_K + qk0).  Lanes past the end repeat the last charge without storing
    // anything, so that the warp does not diverge (a warp with a diverged tail was seen to end
    // several microseconds after the others).
    const bool on = i < n;
    const int ic = on ? i : n - 1;
    const long long gi = S.chg + perm[S.chg + ic];
    const long long sr = S.src + ic, sk = S.src + n + ic;
    const float4 h = xs[2 * gi], l = xs[2 * gi + 1];
    const df X = df_make(h.x, l.x), Y = df_make(h.y, l.y), Z = df_make(h.z, l.z), Q = df_make(h.w, l.w);
    if (on) {
      iperm[gi] = i;
      src_hi[sr] = make_float4(h.x, h.y, h.z, (df_make(S.f_kc.x, S.f_kc.y) * Q).hi);
      src_lo[sr] = make_float4(l.x, l.y, l.z, 0.f);
      bmin[0] = bmax[0] = h.x;
      bmin[1] = bmax[1] = h.y;
      bmin[2] = bmax[2] = h.z;
    }
    const df r2 = X * X + Y * Y + Z * Z;
    // centre test of the FP32 path (k_moment_prep makes the same one), on r = sqrt(r^2) (to
    // within the rounding of r^2)
    const bool centre = r2.hi <= S.f_rc2 && sqrt(df_to_double(r2)) <= kCentreRel * S.a;
    const df s = df_make(S.f_a2.x, S.f_a2.y) * df_recip(r2);
    const df kx = s * X, ky = s * Y, kz = s * Z;
    const df rK = df_make(S.f_a.x, S.f_a.y) * df_sqrt(s);
    const df QK = Q * (df_make(S.f_qk1.x, S.f_qk1.y) * rK + df_make(S.f_qk0.x, S.f_qk0.y));
    // weights of the transposed Kelvin term of the symmetric pair sum (k_pairs_f32.cuh): by
    // Kelvin inversion |x_j - x_i*| = |x_i - x_j*| |x_j| / |x_i|, so charge j's term from i's
    // image is (q_K,i |x_i|) (1 / |x_i - x_j*|) (1 / |x_j|); the real record carries
    // q_K,i |x_i|, the Kelvin record 1 / |x_j|
    const df rr = df_sqrt(r2);
    if (on) {
      if (centre) {
        // image at infinity (its constant potential is added by the moment rows): a zero-strength
        // record, left out of the box; its scale 1e15 / a turns 1 / |x_i - record| (the record
        // sits at 1e15 a) into the limit 1 / a^2 of |x_i| / (|x_j| |x_i - x_j*|) at x_j -> 0
        src_hi[sk] = make_float4((float)(1e15 * S.a), 0.f, 0.f, 0.f);
        src_lo[sk] = make_float4(0.f, 0.f, 0.f, (float)(1e15 * S.inv_a));
        src_lo[sr].w = 0.f;
      } else {
        src_hi[sk] = make_float4(kx.hi, ky.hi, kz.hi, QK.hi);
        src_lo[sk] = make_float4(kx.lo, ky.lo, kz.lo, df_recip(rr).hi);
        src_lo[sr].w = (QK * rr).hi;
        bmin[3] = bmax[3] = kx.hi;
        bmin[4] = bmax[4] = ky.hi;
        bmin[5] = bmax[5] = kz.hi;
      }
    }
  }
  if (prec != HSMA_FP64) {
#pragma unroll
    for (int d = 0; d < 6; ++d)
      for (int o = 16; o > 0; o >>= 1) {
        bmin[d] = fminf(bmin[d], __shfl_xor_sync(0xffffffffu, bmin[d], o));
        bmax[d] = fmaxf(bmax[d], __shfl_xor_sync(0xffffffffu, bmax[d], o));
      }
    if (lane == 0 && i < n) {
      const long long b = S.bb + i / kBox;
      const long long bk = b + (n + kBox - 1) / kBox;
      boxes[2 * b] = make_float4(bmin[0], bmin[1], bmin[2], 0.f);
      boxes[2 * b + 1] = make_float4(bmax[0], bmax[1], bmax[2], 0.f);
      boxes[2 * bk] = make_float4(bmin[3], bmin[4], bmin[5], 0.f);
      boxes[2 * bk + 1] = make_float4(bmax[3], bmax[4], bmax[5], 0.f);
    }
  }
}

void launch_images(const SysDev* sys, const int2* items, int nitems, const double* xyz, const double* q,
                   const float4* xs, const int* perm, int* iperm, float4* src_hi, float4* src_lo, dbl4* src64,
                   float4* boxes, int prec, int* status, cudaStream_t st)
{
  if (nitems <= 0) return;
  launch_k(k_images, nitems * kImgSplit, kImgThreads, 0, st, true, sys, items, xyz, q, xs, perm, iperm, src_hi,
           src_lo, src64, boxes, prec, status);
}

// Moment inputs of one charge in double-float: u, v, w = x/a, rho^2 = |x|^2/a^2, q and q c with
// c = dbar (R_tau r/a^2 - 1)/2, from the (hi, lo) splits of x, y, z, q (FP32 arithmetic only:
// this GPU issues FP64 arithmetic at a small fraction of the FP32 rate).
struct MomentInputs {
  df u, v, w, rho2, q, qc;
};
__device__ __forceinline__ MomentInputs moment_inputs_df(const SysDev& S, df x, df y, df z, df qi)
{
  MomentInputs r;
  const df ia = df_make(S.f_inv_a.x, S.f_inv_a.y);
  r.u = x * ia;
  r.v = y * ia;
  r.w = z * ia;
  r.rho2 = r.u * r.u + r.v * r.v + r.w * r.w;
  r.q = qi;
  const df rr = r.rho2.hi > 0.f ? df_sqrt(r.rho2) : df_make(0.f, 0.f);
  const df c = df_make(S.f_hdbar.x, S.f_hdbar.y) * (df_make(S.f_Rt_a.x, S.f_Rt_a.y) * rr - df_make(1.f, 0.f));
  r.qc = r.q * c;
  return r;
}

// Charge moments of the correction coefficients.  Thread t of a block prepares charge c0 + t:
// the centre constant of a charge at the centre, and its moment inputs u, v, w = x/a, rho^2, q
// and q c in the moment arithmetic R (shared memory), so the moment phase runs on R alone: per
// group of G <= 32 charges, the weights q (M_n - gamma) - q c of every (charge, n), warp w
// computes the column pairs j = w, w + kMomWarps, ... of every charge (lane = charge;
// solid_pair), then thread t accumulates coefficients t + j kMomThreads over the group.  Rows
// are stored as R values in 8-byte slots; slot P holds the block's centre constant.
template <int MAXJ, class R>
__global__ __launch_bounds__(kMomThreads) void k_moments(const SysDev* __restrict__ sys, const int2* __restrict__ items,
                                                         const InDesc* __restrict__ in,
                                                         const double* __restrict__ Mn, Tables tab,
                                                         double* __restrict__ mom, int mom_stride, int G)
{
  extern __shared__ double sm[];
  const double* __restrict__ xyz = in->xyz;
  const double* __restrict__ q = in->q;
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int n = S.n, P = S.P, p = S.p;
  const double dbar = S.dbar, inv_a = S.inv_a;
  const int c0 = it.y * S.mom_tile;
  const int cnt = min(n, c0 + S.mom_tile) - c0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

  static_assert(sizeof(R) == sizeof(double), "moment arithmetic uses 8-byte values");
  static_assert(!Num<R>::is_df, "the FP32 path forms its moments in k_moment_units");
  R* T = reinterpret_cast<R*>(sm);  // [G][P]
  R* cu = T + (size_t)G * P;        // per charge of the tile: u, v, w, rho^2, q, q c
  R* cv = cu + kMomThreads;
  R* cw = cv + kMomThreads;
  R* cr2 = cw + kMomThreads;
  R* cq = cr2 + kMomThreads;
  R* cqc = cq + kMomThreads;
  double* red = reinterpret_cast<double*>(cqc + kMomThreads);  // [kMomWarps]
  const int np1 = tab.pmax + 1;
  R* mg = reinterpret_cast<R*>(red + kMomWarps);  // [pmax + 1] M_n - gamma
  R* wq = mg + np1;                               // [G][pmax + 1] q (M_n - gamma - c) of the group

  // the tile's charges are loaded first (the longest chain of dependent loads: item, system,
  // charges), the recurrence tables beside them
  double x = 0.0, y = 0.0, z = 0.0, qi = 0.0;
  if (tid < cnt) {
    const long long gi = S.chg + c0 + tid;
    x = xyz[3 * gi];
    y = xyz[3 * gi + 1];
    z = xyz[3 * gi + 2];
    qi = q[gi];
  }
  // the recurrence tables in shared memory when they are small (a global load per recurrence
  // step otherwise); visible after the __syncthreads that follows the preparation pass
  const R* ra = Num<R>::is_df ? reinterpret_cast<const R*>(tab.rec_a2) : reinterpret_cast<const R*>(tab.rec_a);
  const R* rb = Num<R>::is_df ? reinterpret_cast<const R*>(tab.rec_b2) : reinterpret_cast<const R*>(tab.rec_b);
  const R* sp = Num<R>::is_df ? reinterpret_cast<const R*>(tab.sprod2) : reinterpret_cast<const R*>(tab.sprod);
  {
    const int pm = tab.pmax;
    const int ntri = (pm + 1) * (pm + 2) / 2;
    if (2 * (size_t)ntri + pm + 1 <= kMomTableSlots) {
      R* tb = wq + (size_t)G * np1;
      for (int i = tid; i < ntri; i += kMomThreads) {
        const R va = ra[i], vb = rb[i], vs = i <= pm ? sp[i] : Num<R>::zero();
        tb[i] = va;
        tb[ntri + i] = vb;
        if (i <= pm) tb[2 * ntri + i] = vs;
      }
      ra = tb;
      rb = tb + ntri;
      sp = tb + 2 * ntri;
    }
  }

  double r0 = 0.0;
  if (tid < cnt) {
    const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
    const double rc = kCentreRel * S.a;
    if (r2 <= 4.0 * rc * rc && sqrt(r2) <= rc) r0 += S.kc_a * qi * (S.gam - 0.5 * dbar);
    const double r = sqrt(r2);
    const double ux = x * inv_a, uy = y * inv_a, uz = z * inv_a;
    cu[tid] = Num<R>::from(ux);
    cv[tid] = Num<R>::from(uy);
    cw[tid] = Num<R>::from(uz);
    cr2[tid] = Num<R>::from(ux * ux + uy * uy + uz * uz);
    cq[tid] = Num<R>::from(qi);
    cqc[tid] = Num<R>::from(qi * (dbar * (S.Rt_a * (r * inv_a) - 1.0) * 0.5));
  }
  if (tid <= p) mg[tid] = Num<R>::from(Mn[S.mn + tid] - S.gam);
  // block sum of the centre-charge constants (fixed order), reduced only when some charge of
  // the tile sits at the centre (FP64 shuffles in every warp cost more than the tile's prep)
  double* out = mom + (size_t)(S.mom + it.y) * mom_stride;
  if (__syncthreads_or(r0 != 0.0)) {
    for (int o = 16; o > 0; o >>= 1) r0 += __shfl_xor_sync(0xffffffffu, r0, o);
    if (lane == 0) red[warp] = r0;
    __syncthreads();
    if (tid == 0) {
      double s = 0.0;
      for (int w = 0; w < kMomWarps; ++w) s += red[w];
      out[P] = s;
    }
  } else if (tid == 0) {
    out[P] = 0.0;
  }
  // the block's rows of A'_nm / (k/(eps1 a)) = sum_i q_i (M_n - gamma - c_i) T_nm(x_i)
  // (the moments (M_n - gamma) U_nm - V_nm with one accumulation per coefficient and charge:
  // the weight of (n, charge) is formed once per group)
  R acc[MAXJ];
  int nidx[MAXJ];
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) {
    acc[j] = Num<R>::zero();
    const int idx = tid + j * kMomThreads;
    int nn = (int)sqrtf((float)idx);
    while (nn * nn > idx) --nn;
    while ((nn + 1) * (nn + 1) <= idx) ++nn;
    nidx[j] = nn;
  }
  // warp w computes the column pairs j = w, w + kMomWarps, ... and lane l charge l of the group
  // (G <= 32): the lanes of a warp run the same chains, without divergence
  const int npair = p / 2 + 1;
  for (int g0 = 0; g0 < cnt; g0 += G) {
    const int gcount = min(G, cnt - g0);
    for (int k = tid; k < gcount * (p + 1); k += kMomThreads) {
      const int g = k / (p + 1), nn = k - g * (p + 1);
      wq[g * np1 + nn] = Num<R>::mul_sub(cq[g0 + g], mg[nn], Num<R>::one(), cqc[g0 + g]);
    }
    if (lane < gcount) {
      const int c = g0 + lane;
      for (int j = warp; j < npair; j += kMomWarps)
        solid_pair<R>(j, p, cu[c], cv[c], cw[c], cr2[c], ra, rb, sp, T + (size_t)lane * P);
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < MAXJ; ++j) {
      const int idx = tid + j * kMomThreads;
      if (idx < P) {
        R u = acc[j];
        for (int g = 0; g < gcount; ++g) u = Num<R>::acc(u, wq[g * np1 + nidx[j]], T[(size_t)g * P + idx]);
        acc[j] = Num<R>::norm(u);
      }
    }
    __syncthreads();
  }
  // the coefficient kernel may launch once every moment block is here: earlier, its CTAs would
  // hold SM resources (waiting) that the order and the records need beside this kernel
  allow_dependents();
#pragma unroll
  for (int j = 0; j < MAXJ; ++j) {
    const int idx = tid + j * kMomThreads;
    if (idx < P) Num<R>::st(out, idx, acc[j]);
  }
}

// Charges per moment group: at most 32 (a warp's lanes) and the group's G (P + pmax + 1) values
// within the shared-memory budget.
static size_t moment_table_slots(int pmax)
{
  const size_t s = 2 * (size_t)(pmax + 1) * (pmax + 2) / 2 + (size_t)(pmax + 1);
  return s <= kMomTableSlots ? s : 0;
}

// blocks_per_sm = 2 halves the budget, so that two blocks (20 warps) share an SM: more warps to
// hide the dependent double-float chains when there are many more blocks than SMs.
int moment_smem_group(int maxP, int blocks_per_sm)
{
  int pmax = (int)std::lround(std::sqrt((double)maxP)) - 1;
  if (pmax < 0) pmax = 0;
  const size_t fixed = (6 * (size_t)kMomThreads + kMomWarps + (pmax + 1) + moment_table_slots(pmax)) * sizeof(double);
  const size_t budget = blocks_per_sm >= 2 ? 112 * 1024 : 192 * 1024;
  int G = 32;  // one warp lane per charge of the group
  const size_t per = ((size_t)maxP + pmax + 1) * sizeof(double);
  const int Gs = budget > fixed ? (int)((budget - fixed) / per) : 0;
  if (G > Gs) G = Gs;
  if (G < 1) G = 1;
  return G;
}

static size_t moment_smem_bytes(int maxP, int G)
{
  int pmax = (int)std::lround(std::sqrt((double)maxP)) - 1;
  if (pmax < 0) pmax = 0;
  return ((size_t)G * (maxP + pmax + 1) + 6 * (size_t)kMomThreads + kMomWarps + (pmax + 1) +
          moment_table_slots(pmax)) *
         sizeof(double);
}

template <int MAXJ>
static void launch_mom(const SysDev* sys, const int2* items, int nitems, int maxP, int G, const InDesc* in,
                       const double* Mn, Tables tab, int prec, double* mom, int mom_stride, cudaStream_t st)
{
  const size_t smem = moment_smem_bytes(maxP, G);
  (void)prec;  // FP64 only (the FP32 path: launch_moment_prep, launch_moment_units)
  launch_k(k_moments<MAXJ, double>, nitems, kMomThreads, smem, st, false, sys, items, in, Mn, tab, mom, mom_stride, G);
}

void launch_moments(const SysDev* sys, const int2* items, int nitems, int maxP, int G, const InDesc* in,
                    const double* Mn, Tables tab, int prec, double* mom, int mom_stride, cudaStream_t st)
{
  if (nitems <= 0) return;
  const int J = (maxP + kMomThreads - 1) / kMomThreads;
  if (J <= 1)
    launch_mom<1>(sys, items, nitems, maxP, G, in, Mn, tab, prec, mom, mom_stride, st);
  else if (J <= 2)
    launch_mom<2>(sys, items, nitems, maxP, G, in, Mn, tab, prec, mom, mom_stride, st);
  else if (J <= 4)
    launch_mom<4>(sys, items, nitems, maxP, G, in, Mn, tab, prec, mom, mom_stride, st);
  else if (J <= 8)
    launch_mom<8>(sys, items, nitems, maxP, G, in, Mn, tab, prec, mom, mom_stride, st);
  else if (J <= 16)
    launch_mom<16>(sys, items, nitems, maxP, G, in, Mn, tab, prec, mom, mom_stride, st);
  else
    launch_mom<26>(sys, items, nitems, maxP, G, in, Mn, tab, prec, mom, mom_stride, st);
}

// ---------------------------------------------------------------------------------------
// FP32 path: the moment rows in double-float, lane = charge.  The unnormalised column chains
// share nothing between charges, so a warp takes 32 charges of one column pair and forms the
// 32 charges' terms of each coefficient side by side, then sums them across the lanes with a
// transposed warp reduction; no shared memory and no block barrier, every lane busy.
//
// k_moment_prep, a quad of kMomPrepSplit lanes per charge: the inputs that every column of the
// charge reuses.  Quad lane k splits input k of the charge (x, y, z, q; split_double) and the
// quad shares the splits; then lane k writes the powers z^m and the weights of degree n for
// m, n = k mod 4 (z^m = z^k (z^4)^s), a quarter of the sequential chain of complex products.
__global__ __launch_bounds__(kMomPrepThreads) void k_moment_prep(const SysDev* __restrict__ sys,
                                                                 const int2* __restrict__ items,
                                                                 const InDesc* __restrict__ inp,
                                                                 const double* __restrict__ Mn,
                                                                 float4* __restrict__ geo, float4* __restrict__ mz,
                                                                 float2* __restrict__ mwq, double* __restrict__ mcen)
{
  static_assert(kMomPrepThreads > HSMA_P_MAX, "one thread per degree for M_n - gamma");
  static_assert(kMomPrepSplit == 4, "a quad per charge: x, y, z, q and z^k, k < 4");
  __shared__ df smg[kMomPrepThreads];  // M_n - gamma
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int ns = S.n, p = S.p;
  const int lane = threadIdx.x & 31, sub = lane & 3, quad = lane & ~3;
  const int i = it.y * kMomPrepCharges + (int)threadIdx.x / kMomPrepSplit;
  const bool live = i < ns;
  const long long gi = S.chg + (live ? i : 0);
  double xin = 0.0;
  if (live) xin = sub < 3 ? inp->xyz[3 * gi + sub] : inp->q[gi];
  if ((int)threadIdx.x <= p) smg[threadIdx.x] = df_from_double(Mn[S.mn + threadIdx.x] - S.gam);
  // every block of the grid is resident once this is reached: the unit kernel's blocks may
  // start (they wait for this grid's writes before reading them)
  allow_dependents();
  const df dv = df_from_double(xin);
  df in[4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
    in[k] = df_make(__shfl_sync(0xffffffffu, dv.hi, quad + k), __shfl_sync(0xffffffffu, dv.lo, quad + k));
  const double qv = __shfl_sync(0xffffffffu, xin, quad + 3);
  __syncthreads();
  if (!live) return;
  const MomentInputs mi = moment_inputs_df(S, in[0], in[1], in[2], in[3]);
  if (sub == 0) {
    // the centre constant of a charge whose image is at infinity, by the FP32 path's centre
    // test of k_images on the same splits (FP64 only near the centre)
    const df r2 = in[0] * in[0] + in[1] * in[1] + in[2] * in[2];
    const bool centre = r2.hi <= S.f_rc2 && sqrt(df_to_double(r2)) <= kCentreRel * S.a;
    mcen[gi] = centre ? S.kc_a * qv * (S.gam - 0.5 * S.dbar) : 0.0;
    geo[gi] = make_float4(2.f * mi.w.hi, 2.f * mi.w.lo, mi.rho2.hi, mi.rho2.lo);
  }
  // z^2, z^4 and z^sub
  const df uv = mi.u * mi.v;
  const df u2r = df_mul_sub(mi.u, mi.u, mi.v, mi.v), u2i = df_make(2.f * uv.hi, 2.f * uv.lo);
  const df rs = u2r * u2i;
  const df u4r = df_mul_sub(u2r, u2r, u2i, u2i), u4i = df_make(2.f * rs.hi, 2.f * rs.lo);
  df zr = df_make(1.f, 0.f), zi = df_make(0.f, 0.f);
  if (sub == 1) {
    zr = mi.u;
    zi = mi.v;
  } else if (sub == 2) {
    zr = u2r;
    zi = u2i;
  } else if (sub == 3) {
    zr = df_mul_sub(u2r, mi.u, u2i, mi.v);
    zi = df_mul_sub(u2r, mi.v, -u2i, mi.u);
  }
  const long long zb = S.mzo + i;
  for (int m = sub; m <= p; m += kMomPrepSplit) {
    mz[zb + (long long)m * ns] = make_float4(zr.hi, zr.lo, zi.hi, zi.lo);
    const df nr = df_mul_sub(zr, u4r, zi, u4i);
    const df ni = df_mul_sub(zr, u4i, -zi, u4r);
    zr = nr;
    zi = ni;
  }
  for (int n = sub; n <= p; n += kMomPrepSplit) {
    const df wq = df_mul_sub(mi.q, smg[n], df_make(1.f, 0.f), mi.qc);
    mwq[zb + (long long)n * ns] = make_float2(wq.hi, wq.lo);
  }
}

// a + b with the low parts summed, not renormalised (the caller renormalises once)
__device__ __forceinline__ df df_add_lazy(df a, df b)
{
  const df s = two_sum(a.hi, b.hi);
  return df_make(s.hi, s.lo + (a.lo + b.lo));
}

__device__ __forceinline__ df shfl_xor_df(df v, int o)
{
  return df_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

// One level of the transposed reduction: lanes with bit H of the lane set keep the upper half
// of the H-pair window of v and send the lower half to the partner lane ^ H (and vice versa).
template <int H>
__device__ __forceinline__ void treduce_level(df* v, bool upper)
{
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const df keep = upper ? v[H + k] : v[k];
    const df send = upper ? v[k] : v[H + k];
    v[k] = df_add_lazy(keep, shfl_xor_df(send, 2 * H));
  }
}

// Sum over the 32 lanes of each of the 16 values v[0..15] of a lane: afterwards lane l holds
// the sum of value (l >> 1) & 15 (lanes l and l ^ 1 the same) in v[0], renormalised.  Fixed
// order: the result does not depend on scheduling.
__device__ __forceinline__ df warp_treduce16(df* v, int lane)
{
  treduce_level<8>(v, (lane & 16) != 0);
  treduce_level<4>(v, (lane & 8) != 0);
  treduce_level<2>(v, (lane & 4) != 0);
  treduce_level<1>(v, (lane & 2) != 0);
  return df_norm(df_add_lazy(v[0], shfl_xor_df(v[0], 1)));
}

// Steps n = n0 .. n0 + NS - 1 of one column chain for the lane's charge: values 2k, 2k + 1 are
// the real and sine parts of q (M_n - gamma - c) S_n z^m for n = n0 + k (zero past n = p and for
// a dead lane), then the chain advances, S_{n+1} = 2 w S_n - beta_{n+1,m} rho^2 S_{n-1}.  On
// entry qa = S_n0, qb = S_{n0-1}, tb = table index of (n0 + 1, m), wp = the weight of degree n0
// (next degree: + ns).  A chain may run up to NS - 1 steps past p (beta is padded for that).
template <int NS>
__device__ __forceinline__ void moment_chain_steps(df W, df R2, df& qa, df& qb, int n0, int p, int& tb,
                                                   const float2* __restrict__ beta,
                                                   const float2* __restrict__ wp, long long ns, bool live,
                                                   float4 z, df* v)
{
#pragma unroll
  for (int k = 0; k < NS; ++k) {
    const int n = n0 + k;
    const float2 wv = (live && n <= p) ? wp[k * ns] : make_float2(0.f, 0.f);
    const df t = df_mul_lazy(df_make(wv.x, wv.y), qa);
    v[2 * k] = df_mul_lazy(t, df_make(z.x, z.y));
    v[2 * k + 1] = df_mul_lazy(t, df_make(z.z, z.w));
    const float2 bt = beta[tb];
    const df nx = df_mul_sub(W, qa, df_mul_lazy(df_make(bt.x, bt.y), R2), qb);
    qb = qa;
    qa = nx;
    tb += n + 2;
  }
}

// k_moment_units: the unit's columns m1 = j and m2 = p - j (n = m..p each; one column when they
// coincide) in batches of kMomUnitSteps steps, 16 values per lane that warp_treduce16 sums over
// the lanes.  The first nA batches take 4 steps of each column (the shorter column m2 is done
// after them), the next nB batches 8 steps of column m1 alone: every step of a batch has a
// fixed column and degree offset, with no per-step selection.  The running sum of a batch's
// values over the tile's groups of 32 charges stays in the warp's shared memory (lane l: value
// (l >> 1) & 15).  The chain runs on S_n = T_nm / (e_nm sprod_m z^m) (k_setup), and the row value
// is the sum times e_nm sprod_m (mnrm2).
constexpr int kMomUnitMaxBatches = 11;  // nA + nB for every p <= HSMA_P_MAX and pair j
static_assert(HSMA_P_MAX <= 80, "kMomUnitMaxBatches is the largest nA + nB for p <= 80");
struct MomentUnitShape {
  int m1, m2, nA, nB;
};
__device__ __forceinline__ MomentUnitShape moment_unit_shape(int p, int j)
{
  MomentUnitShape u;
  u.m1 = j;
  u.m2 = p - j;
  const int L1 = p - u.m1 + 1, L2 = u.m2 != u.m1 ? p - u.m2 + 1 : 0;
  u.nA = (L2 + 3) / 4;
  const int R = L1 - 4 * u.nA;
  u.nB = R > 0 ? (R + 7) / 8 : 0;
  return u;
}
// column and degree of value k (0..7 steps) of batch b
__device__ __forceinline__ void moment_unit_value(const MomentUnitShape& u, int b, int k, int& m, int& n)
{
  if (b < u.nA) {
    m = k < 4 ? u.m1 : u.m2;
    n = m + 4 * b + (k & 3);
  } else {
    m = u.m1;
    n = u.m1 + 4 * u.nA + 8 * (b - u.nA) + k;
  }
}

__global__ __launch_bounds__(kMomUnitWarps * 32, 24 / kMomUnitWarps) void k_moment_units(
    const SysDev* __restrict__ sys, const int2* __restrict__ units, int nunits, const float4* __restrict__ geo,
    const float4* __restrict__ mz, const float2* __restrict__ mwq, const double* __restrict__ mcen, Tables tab,
    double* __restrict__ mom, int mom_stride)
{
  static_assert(kMomUnitSteps == 8, "mode A: 4 + 4 steps, mode B: 8 steps");
  __shared__ float2 sacc[kMomUnitWarps][kMomUnitMaxBatches][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int u = blockIdx.x * kMomUnitWarps + warp;
  if (u >= nunits) return;
  const int2 it = units[u];
  const SysDev& S = sys[it.x];
  const int ns = S.n, p = S.p;
  const int tile = it.y >> 7, j = it.y & 127;
  const MomentUnitShape sh = moment_unit_shape(p, j);
  const int nbat = sh.nA + sh.nB;
  const int cb = tile * S.mom_tile, ce = min(ns, cb + S.mom_tile);
  const float2* __restrict__ beta = tab.mbeta2;
  float2* acc = &sacc[warp][0][lane];  // acc[32 b]: batch b
  for (int b = 0; b < nbat; ++b) acc[32 * b] = make_float2(0.f, 0.f);
  grid_dependency_wait();  // the prep's tables

  double cen = 0.0;
  for (int c0 = cb; c0 < ce; c0 += 32) {
    const int i = c0 + lane;
    const bool live = i < ce;
    const long long zb = S.mzo + i;
    const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 g = live ? geo[S.chg + i] : zero4;
    const float4 z1 = live ? mz[zb + (long long)sh.m1 * ns] : zero4;
    const float4 z2 = live && sh.nA > 0 ? mz[zb + (long long)sh.m2 * ns] : zero4;
    if (j == 0 && live) cen += mcen[S.chg + i];
    const df W = df_make(g.x, g.y), R2 = df_make(g.z, g.w);
    // chain states: S_n, S_{n-1} at the next step's degree, and that degree's table index + 1 row
    df qa1 = df_make(1.f, 0.f), qb1 = df_make(0.f, 0.f), qa2 = df_make(1.f, 0.f), qb2 = df_make(0.f, 0.f);
    int tb1 = (sh.m1 + 1) * (sh.m1 + 2) / 2 + sh.m1, tb2 = (sh.m2 + 1) * (sh.m2 + 2) / 2 + sh.m2;
    const float2* wp1 = mwq + zb + (long long)sh.m1 * ns;
    const float2* wp2 = mwq + zb + (long long)sh.m2 * ns;
#pragma unroll 1
    for (int b = 0; b < sh.nA; ++b) {
      df v[16];
      moment_chain_steps<4>(W, R2, qa1, qb1, sh.m1 + 4 * b, p, tb1, beta, wp1 + 4LL * b * ns, ns, live, z1, v);
      moment_chain_steps<4>(W, R2, qa2, qb2, sh.m2 + 4 * b, p, tb2, beta, wp2 + 4LL * b * ns, ns, live, z2, v + 8);
      const df r = warp_treduce16(v, lane);
      const float2 a = acc[32 * b];
      const df sum = df_make(a.x, a.y) + r;
      acc[32 * b] = make_float2(sum.hi, sum.lo);
    }
    const int n1 = sh.m1 + 4 * sh.nA;
#pragma unroll 1
    for (int b = 0; b < sh.nB; ++b) {
      df v[16];
      moment_chain_steps<8>(W, R2, qa1, qb1, n1 + 8 * b, p, tb1, beta, wp1 + (4LL * sh.nA + 8LL * b) * ns, ns,
                            live, z1, v);
      const df r = warp_treduce16(v, lane);
      const float2 a = acc[32 * (sh.nA + b)];
      const df sum = df_make(a.x, a.y) + r;
      acc[32 * (sh.nA + b)] = make_float2(sum.hi, sum.lo);
    }
  }
  // the coefficient kernel may launch once every unit is here
  allow_dependents();
  double* out = mom + (size_t)(S.mom + tile) * mom_stride;
  if ((lane & 1) == 0) {
    const int part = (lane >> 1) & 1;  // 0: cosine (real) part, 1: sine part
    for (int b = 0; b < nbat; ++b) {
      int m, n;
      moment_unit_value(sh, b, lane >> 2, m, n);
      if (n <= p && !(part && m == 0)) {
        const float2 f = tab.mnrm2[n * (n + 1) / 2 + m];
        const float2 a = acc[32 * b];
        const df val = df_make(a.x, a.y) * df_make(f.x, f.y);
        reinterpret_cast<float2*>(out)[n * n + n + (part ? -m : m)] = make_float2(val.hi, val.lo);
      }
    }
  }
  if (j == 0) {
    for (int o = 16; o > 0; o >>= 1) cen += __shfl_xor_sync(0xffffffffu, cen, o);
    if (lane == 0) out[S.P] = cen;
  }
}

void launch_moment_prep(const SysDev* sys, const int2* items, int nitems, const InDesc* in, const double* Mn,
                        float4* geo, float4* mz, float2* mwq, double* mcen, cudaStream_t st)
{
  if (nitems <= 0) return;
  launch_k(k_moment_prep, nitems, kMomPrepThreads, 0, st, false, sys, items, in, Mn, geo, mz, mwq, mcen);
}

void launch_moment_units(const SysDev* sys, const int2* units, int nunits, const float4* geo,
                         const float4* mz, const float2* mwq, const double* mcen, Tables tab, double* mom,
                         int mom_stride, cudaStream_t st)
{
  if (nunits <= 0) return;
  const int grid = (nunits + kMomUnitWarps - 1) / kMomUnitWarps;
  launch_pdl(k_moment_units, grid, kMomUnitWarps * 32, 0, st, sys, units, nunits, geo, mz, mwq, mcen, tab, mom,
             mom_stride);
}

// ---------------------------------------------------------------------------------------
// hat A'_nm = (k/(eps1 a)) [(M_n - gamma) U_nm - V_nm] = (k/(eps1 a)) sum over the moment rows
// (each row holds sum_i q_i (M_n - gamma - c_i) T_nm(x_i/a) over its block's charges).  A block
// owns kCoefChunk coefficients (one per lane); its kCoefWarps warps split the rows (warp w takes
// rows w, w + kCoefWarps, ...), and warp 0 adds the warp sums in order, so the result does not
// depend on scheduling.  Sums run in the moment arithmetic R; the coefficient is formed in FP64
// and also stored as an FP32 (hi, lo) pair for the FP32 path's surface synthesis.
constexpr int kCoefWarps = 8;  // 256-thread blocks: they fit beside a pair launch that leaves a CTA slot free
template <class R>
__global__ __launch_bounds__(kCoefWarps * 32) void k_coef_reduce(const SysDev* __restrict__ sys,
                                                                 const int2* __restrict__ items,
                                                                 const double* __restrict__ mom, int mom_stride,
                                                                 const double* __restrict__ Mn,
                                                                 double* __restrict__ coef, float2* __restrict__ coef2,
                                                                 double* __restrict__ r0)
{
  __shared__ R su[kCoefWarps][kCoefChunk];
  __shared__ double sr[kCoefWarps];
  __shared__ float2 srd[kCoefWarps];
  // the item and its system are read before the wait for the moment rows
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int P = S.P, nb = S.mom_blocks;
  const double kc_a = S.kc_a;
  const double* base = mom + (size_t)S.mom * mom_stride;
  grid_dependency_wait();  // the moment rows
  allow_dependents();      // (the surface kernel's CTAs wait only while this kernel works)
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int idx = it.y * kCoefChunk + lane;
  R U = Num<R>::zero();
  double Rs = 0.0;
  if (idx < P) {
    // rows b = warp, warp + kCoefWarps, ... in ascending order, twelve rows' loads in flight
    constexpr int kRows = 12;
    for (int b0 = warp; b0 < nb; b0 += kRows * kCoefWarps) {
      R u[kRows];
#pragma unroll
      for (int k = 0; k < kRows; ++k) {
        const int b = b0 + k * kCoefWarps;
        u[k] = b < nb ? Num<R>::ld(base, (long long)b * mom_stride + idx) : Num<R>::zero();
      }
#pragma unroll
      for (int k = 0; k < kRows; ++k)
        if (b0 + k * kCoefWarps < nb) U = U + u[k];
    }
  }
  // the rows' centre constants (block 0): thread t takes rows t, t + kCoefWarps 32, ... (all
  // loads of the block in flight at once), then a fixed-order reduction over the lanes and the
  // warps; the FP32 path sums in double-float (FP64 additions of a whole block would queue on one
  // SM's FP64 unit)
  df Rsd = df_make(0.f, 0.f);
  if (it.y == 0) {
    for (int b = threadIdx.x; b < nb; b += kCoefWarps * 32) {
      const double v = base[(size_t)b * mom_stride + P];
      if (Num<R>::is_df)
        Rsd = Rsd + df_from_double(v);
      else
        Rs += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      if (Num<R>::is_df)
        Rsd = Rsd + df_make(__shfl_xor_sync(0xffffffffu, Rsd.hi, o), __shfl_xor_sync(0xffffffffu, Rsd.lo, o));
      else
        Rs += __shfl_xor_sync(0xffffffffu, Rs, o);
    }
  }
  su[warp][lane] = U;
  if (lane == 0) {
    sr[warp] = Rs;
    srd[warp] = make_float2(Rsd.hi, Rsd.lo);
  }
  __syncthreads();
  if (warp == 0) {
    U = Num<R>::zero();
#pragma unroll
    for (int w = 0; w < kCoefWarps; ++w) U = U + su[w][lane];
    if (idx < P) {
      const double c = kc_a * Num<R>::to(U);
      coef[S.coef + idx] = c;
      coef2[S.coef + idx] = pair_of(c);
    }
    if (it.y == 0 && lane == 0) {
      if (Num<R>::is_df) {
        df t = df_make(0.f, 0.f);
        for (int w = 0; w < kCoefWarps; ++w) t = t + df_make(srd[w].x, srd[w].y);
        r0[it.x] = df_to_double(t);
      } else {
        double t = 0.0;
        for (int w = 0; w < kCoefWarps; ++w) t += sr[w];
        r0[it.x] = t;
      }
    }
  }
}

void launch_coef_reduce(const SysDev* sys, const int2* items, int nitems, const double* mom, int mom_stride,
                        const double* Mn, double* coef, float2* coef2, double* r0, int prec, cudaStream_t st)
{
  if (nitems <= 0) return;
  if (prec == HSMA_FP64)
    launch_pdl(k_coef_reduce<double>, nitems, kCoefWarps * 32, 0, st, sys, items, mom, mom_stride, Mn, coef, coef2,
               r0);
  else
    launch_pdl(k_coef_reduce<df>, nitems, kCoefWarps * 32, 0, st, sys, items, mom, mom_stride, Mn, coef, coef2, r0);
}

// ---------------------------------------------------------------------------------------
// Surface images (Green's second identity + central difference, eq. threeintegrals) from
//   Phi = sum A'_nm T_nm(y/a),   dPhi/dr = sum n A'_nm T_nm(y/a) / R_tau
// at each Fibonacci point y: monopole Q0 = w dPhi/dr / (4 pi) at y = R_tau yhat and dipole
// D = w Phi / (4 pi) between y_- and y_+.
constexpr int kSurfThreads = 256;
constexpr int kSurfWarps = kSurfThreads / 32;
static_assert(kSurfWarps == kSurfPointsPerBlock, "one warp per surface point");
static_assert(kSurfWarps == kSurfMatWarps, "k_surface_mat blocks of kSurfMatWarps warps");

__device__ __forceinline__ void surface_records(const SysDev& S, long long o, const dbl4& yw, double ph, double dph,
                                                int prec, float4* __restrict__ surf_a, float4* __restrict__ surf_b,
                                                dbl4* __restrict__ surf64_a, double* __restrict__ surf64_b,
                                                double2* __restrict__ surfqd)
{
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

// Solid harmonics of the auxiliary-sphere points, T_nm(y_j/a), once per layout (FP64; one warp
// per point, lane = column).  y_j/a = (1 + tau) yhat_j does not depend on a, so systems with the
// same (tau, M, F1, F2, p) share one table, row j at S.sb + j P; the FP32 path keeps each value
// as an FP32 (hi, lo) pair in its 8-byte slot.
__global__ __launch_bounds__(kSurfThreads) void k_surface_basis(const SysDev* __restrict__ sys,
                                                                const int2* __restrict__ items, Tables tab,
                                                                const dbl4* __restrict__ surfx, double* __restrict__ sb,
                                                                int prec)
{
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j = it.y * kSurfWarps + warp;
  if (j >= S.M) return;
  const dbl4 yw = surfx[S.surf + j];
  const double u = yw.x * S.inv_a, v = yw.y * S.inv_a, w = yw.z * S.inv_a;
  const double rho2 = u * u + v * v + w * w;
  double* row = sb + S.sb + (long long)j * S.P;
  for (int m = lane; m <= S.p; m += 32) solid_column<double>(m, S.p, u, v, w, rho2, tab, row);
  if (prec != HSMA_FP64) {
    __syncwarp();
    for (int i = lane; i < S.P; i += 32) {
      const double x = row[i];
      reinterpret_cast<float2*>(row)[i] = pair_of(x);
    }
  }
}

void launch_surface_basis(const SysDev* sys, const int2* items, int nitems, Tables tab, const dbl4* surfx, double* sb,
                          int prec, cudaStream_t st)
{
  if (nitems <= 0) return;
  k_surface_basis<<<nitems, kSurfThreads, 0, st>>>(sys, items, tab, surfx, sb, prec);
}

// One level of a transposed reduction over the lanes (R arithmetic): lanes with lane bit OFF set
// keep the upper half of the 2H-value window of v and send the lower half to the partner lane
// ^ OFF, the others the reverse.
template <int H, int OFF, class R>
__device__ __forceinline__ void treduce_level_r(R* v, int lane)
{
  const bool upper = (lane & OFF) != 0;
#pragma unroll
  for (int k = 0; k < H; ++k) {
    const R keep = upper ? v[H + k] : v[k];
    const R send = upper ? v[k] : v[H + k];
    v[k] = keep + Num<R>::shfl(send, OFF);
  }
}

// Per step, with the basis: a warp takes PW points (1, 2 or 4), lanes stride the coefficients
// (R arithmetic, PW independent sums of Phi and of n Phi per lane), and the 2 PW sums are added
// over the lanes by one transposed reduction (lane l: sum (l >> (5 - log2(2 PW))) mod 2 PW, in a
// fixed order).  The block stages the coefficients once for its kSurfWarps PW points, and warp 0
// forms the records of all of them (lane = point).  Several points per warp amortise the
// staging and the reduction when there are many blocks; one point per warp gives the most
// blocks (lowest latency) when there are few.
template <int V, class R>
__device__ __forceinline__ void treduce_r(R* v, int lane)
{
  static_assert(V == 2 || V == 4 || V == 8, "2, 4 or 8 sums");
  if (V == 8) {
    treduce_level_r<4, 16>(v, lane);
    treduce_level_r<2, 8>(v, lane);
    treduce_level_r<1, 4>(v, lane);
  } else if (V == 4) {
    treduce_level_r<2, 16>(v, lane);
    treduce_level_r<1, 8>(v, lane);
  } else {
    treduce_level_r<1, 16>(v, lane);
  }
#pragma unroll
  for (int off = 32 / V / 2; off > 0; off >>= 1) v[0] = v[0] + Num<R>::shfl(v[0], off);
}

template <int PW, class R>
__global__ __launch_bounds__(kSurfThreads) void k_surface_mat(const SysDev* __restrict__ sys,
                                                              const int2* __restrict__ items,
                                                              const double* __restrict__ coef,
                                                              const float2* __restrict__ coef2,
                                                              const double* __restrict__ sb,
                                                              float4* __restrict__ surf_a, float4* __restrict__ surf_b,
                                                              dbl4* __restrict__ surf64_a,
                                                              double* __restrict__ surf64_b,
                                                              const dbl4* __restrict__ surfx,
                                                              double2* __restrict__ surfqd, int prec)
{
  constexpr int PTS = kSurfWarps * PW;  // points per block
  extern __shared__ double sm[];
  __shared__ R s_sum[kSurfWarps][2 * PW];  // per warp: Phi of its points, then n Phi
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int P = S.P, M = S.M;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int j0 = it.y * PTS + warp * PW;
  // the basis rows (a layout constant) and, in warp 0, the block's points are loaded before the
  // wait for the coefficients: kRowBatch row loads per point and lane in flight
  constexpr int kRowBatch = 16 / PW;
  const double* row[PW];
  bool live[PW];
#pragma unroll
  for (int t = 0; t < PW; ++t) {
    live[t] = j0 + t < M;
    row[t] = sb + S.sb + (long long)(live[t] ? j0 + t : 0) * P;
  }
  R bv[PW][kRowBatch];
#pragma unroll
  for (int t = 0; t < PW; ++t)
#pragma unroll
    for (int k = 0; k < kRowBatch; ++k) {
      const int i = lane + 32 * k;
      bv[t][k] = live[t] && i < P ? Num<R>::ld(row[t], i) : Num<R>::zero();
    }
  const int jl = it.y * PTS + lane;  // warp 0: the point of lane l < PTS
  dbl4 yw = make_dbl4(0.0, 0.0, 0.0, 0.0);
  if (warp == 0 && lane < PTS && jl < M) yw = surfx[S.surf + jl];

  grid_dependency_wait();  // the coefficients of k_coef_reduce
  R* A = reinterpret_cast<R*>(sm);  // [P] A'_nm
  R* nA = A + P;                    // [P] n A'_nm
  for (int i = threadIdx.x; i < P; i += kSurfThreads) {
    int nn = (int)sqrtf((float)i);
    while (nn * nn > i) --nn;
    while ((nn + 1) * (nn + 1) <= i) ++nn;
    const R c = Num<R>::coefv(coef, coef2, S.coef + i);
    A[i] = c;
    nA[i] = Num<R>::from_int(nn) * c;
  }
  __syncthreads();
  R v[2 * PW];
#pragma unroll
  for (int t = 0; t < 2 * PW; ++t) v[t] = Num<R>::zero();
  for (int i0 = 0;;) {
#pragma unroll
    for (int k = 0; k < kRowBatch; ++k) {
      const int i = i0 + lane + 32 * k;
      if (i < P) {
        const R a = A[i], na = nA[i];
#pragma unroll
        for (int t = 0; t < PW; ++t) {
          v[t] = Num<R>::acc(v[t], a, bv[t][k]);
          v[PW + t] = Num<R>::acc(v[PW + t], na, bv[t][k]);
        }
      }
    }
    i0 += 32 * kRowBatch;
    if (i0 >= P) break;
#pragma unroll
    for (int t = 0; t < PW; ++t)
#pragma unroll
      for (int k = 0; k < kRowBatch; ++k) {
        const int i = i0 + lane + 32 * k;
        bv[t][k] = live[t] && i < P ? Num<R>::ld(row[t], i) : Num<R>::zero();
      }
  }
#pragma unroll
  for (int t = 0; t < 2 * PW; ++t) v[t] = Num<R>::norm(v[t]);
  treduce_r<2 * PW>(v, lane);
  constexpr int sh = PW == 4 ? 2 : (PW == 2 ? 3 : 4);  // lane l holds sum (l >> sh) mod 2 PW
  if ((lane & ((1 << sh) - 1)) == 0) s_sum[warp][lane >> sh] = Num<R>::norm(v[0]);
  __syncthreads();
  // the records of the block's points from one warp (lane l: point l), so that their FP64
  // arithmetic issues once per block rather than once per point
  if (warp == 0 && lane < PTS && jl < M) {
    const int w = lane / PW, t = lane % PW;
    surface_records(S, S.surf + jl, yw, Num<R>::to(s_sum[w][t]), Num<R>::to(s_sum[w][PW + t]), prec, surf_a, surf_b,
                    surf64_a, surf64_b, surfqd);
  }
}

// Without a basis table (too large for the workspace): lane m runs column m of the recurrence
// at the point itself.
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
  grid_dependency_wait();  // the coefficients of k_coef_reduce
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
  if (lane == 0) surface_records(S, o, yw, ph, dph, prec, surf_a, surf_b, surf64_a, surf64_b, surfqd);
}

template <int PW>
static void launch_surface_mat(const int2* items, int nitems, size_t smem, const SysDev* sys, const double* coef,
                               const float2* coef2, const double* sb, float4* surf_a, float4* surf_b,
                               dbl4* surf64_a, double* surf64_b, dbl4* surfx, double2* surfqd, int prec,
                               cudaStream_t st)
{
  if (prec == HSMA_FP64)
    launch_pdl(k_surface_mat<PW, double>, nitems, kSurfThreads, smem, st, sys, items, coef, coef2, sb, surf_a, surf_b,
               surf64_a, surf64_b, surfx, surfqd, prec);
  else
    launch_pdl(k_surface_mat<PW, df>, nitems, kSurfThreads, smem, st, sys, items, coef, coef2, sb, surf_a, surf_b,
               surf64_a, surf64_b, surfx, surfqd, prec);
}

// registers of the largest CTA among the coefficient and surface kernels of a precision (the
// kernels that a real/Kelvin pair launch beside them must leave room for)
int chain_block_regs(int prec)
{
  auto regs = [](const void* f, int threads) {
    cudaFuncAttributes a{};
    cudaFuncGetAttributes(&a, f);
    return (a.numRegs + 7) / 8 * 8 * threads;
  };
  int r = 0;
  if (prec == HSMA_FP64) {
    r = std::max(r, regs((const void*)k_coef_reduce<double>, kCoefWarps * 32));
    r = std::max(r, regs((const void*)k_surface_mat<1, double>, kSurfThreads));
    r = std::max(r, regs((const void*)k_surface_mat<2, double>, kSurfThreads));
    r = std::max(r, regs((const void*)k_surface_mat<4, double>, kSurfThreads));
    r = std::max(r, regs((const void*)k_surface<double>, kSurfThreads));
  } else {
    r = std::max(r, regs((const void*)k_coef_reduce<df>, kCoefWarps * 32));
    r = std::max(r, regs((const void*)k_surface_mat<1, df>, kSurfThreads));
    r = std::max(r, regs((const void*)k_surface_mat<2, df>, kSurfThreads));
    r = std::max(r, regs((const void*)k_surface_mat<4, df>, kSurfThreads));
    r = std::max(r, regs((const void*)k_surface<df>, kSurfThreads));
  }
  return r;
}

void launch_surface(const SysDev* sys, const int2* items, int nitems, int maxP, int pw, const double* coef,
                    const float2* coef2, const double* sb, Tables tab, float4* surf_a, float4* surf_b,
                    dbl4* surf64_a, double* surf64_b, dbl4* surfx, double2* surfqd, int prec, cudaStream_t st)
{
  if (nitems <= 0) return;
  if (sb) {
    const size_t smem = 2 * (size_t)maxP * sizeof(double);
    if (pw == 4)
      launch_surface_mat<4>(items, nitems, smem, sys, coef, coef2, sb, surf_a, surf_b, surf64_a, surf64_b, surfx,
                            surfqd, prec, st);
    else if (pw == 2)
      launch_surface_mat<2>(items, nitems, smem, sys, coef, coef2, sb, surf_a, surf_b, surf64_a, surf64_b, surfx,
                            surfqd, prec, st);
    else
      launch_surface_mat<1>(items, nitems, smem, sys, coef, coef2, sb, surf_a, surf_b, surf64_a, surf64_b, surfx,
                            surfqd, prec, st);
    return;
  }
  const size_t smem = (size_t)maxP * sizeof(double);
  if (prec == HSMA_FP64)
    launch_pdl(k_surface<double>, nitems, kSurfThreads, smem, st, sys, items, coef, tab, surf_a, surf_b, surf64_a,
               surf64_b, surfx, surfqd, prec);
  else
    launch_pdl(k_surface<df>, nitems, kSurfThreads, smem, st, sys, items, coef, tab, surf_a, surf_b, surf64_a,
               surf64_b, surfx, surfqd, prec);
}

template <class R>
static void surface_attrs()
{
  cudaFuncSetAttribute(k_surface<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
  cudaFuncSetAttribute(k_surface_mat<1, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
  cudaFuncSetAttribute(k_surface_mat<2, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
  cudaFuncSetAttribute(k_surface_mat<4, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 128 * 1024);
}

void init_source_kernels()
{
  cudaFuncSetAttribute(k_moments<1, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_moments<2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_moments<4, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_moments<8, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_moments<16, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  cudaFuncSetAttribute(k_moments<26, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  surface_attrs<double>();
  surface_attrs<df>();
}

}  // namespace hsma
