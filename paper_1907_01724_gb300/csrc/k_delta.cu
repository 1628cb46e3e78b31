// Single-charge moves of a Monte Carlo chain: energy change Delta E and the commit of a move.
//
// The paper's method (Sec. 2.4) is linear in the charges: with charge k moved from x_k to x',
// only the terms that involve k change.  With E = E_Coul + E_Kelvin + E_corr,
//   dE_Coul   = q_k sum_{j!=k} k q_j/eps1 (1/|x'-x_j| - 1/|x_k-x_j|)
//   dE_Kelvin = 1/2 sum_{j!=k} [q_k (K_j(x') - K_j(x_k)) + q_j (K'_k(x_j) - K_k(x_j))]
//               + 1/2 q_k (K'_k(x') - K_k(x_k)),
// where K_j(x) = k q_K,j/(eps1 |x - r_K,j|) is the potential of j's modified Kelvin image
// (a constant for a centre charge) and K'_k is k's image after the move.  The correction part
// is E_corr = 1/2 sum_l [Q0_l V0_l + D_l V1_l], where Q0_l, D_l are the monopole/dipole
// strengths of surface point l (linear in the coefficients A) and V0_l = sum_i q_i G0(x_i, y_l),
// V1_l = sum_i q_i G1(x_i, y_l) are the potentials of the real charges under the two surface
// kernels.  The move changes A by a rank-one term dA and V by dV_l = q_k (G(x', y_l) - G(x_k, y_l)):
//   dE_corr = 1/2 sum_l [dQ0_l (V0_l + dV0_l) + Q0_l dV0_l + dD_l (V1_l + dV1_l) + D_l dV1_l].
// The surface strengths of dA follow from the addition theorem without touching all P
// coefficients:  Phi(y; dA) = sum_n a'_n (|x'||y|/a^2)^n P_n(xhat'.yhat) - (same for x_k), with
// a_n = k q_k/(eps1 a) (M_n - gamma - c(x)), c(x) = dbar (R_tau |x|/a^2 - 1)/2 (Sec. 2.4).
// Requests are batched: one launch serves many (system, k, x') requests; every request owns a
// range of work items whose partial sums are added in a fixed order by the last block.
#include <math.h>

#include "df64.cuh"
#include "fp32_pair.cuh"
#include "hsma_internal.cuh"

namespace hsma {

constexpr int kDeltaThreads = kDeltaBlock;


// Kelvin image of a charge (position x, charge q): position, strength k q_K/eps1, or the centre
// constant when |x| <= kCentreRel a.  Same separately rounded operations as k_images_moments.
struct Image {
  double x, y, z, Q, C;  // C: constant potential of a centre charge (then Q = 0)
  bool centre;
};

__device__ __forceinline__ Image kelvin_image(const SysDev& S, double x, double y, double z, double q)
{
  Image im;
  const double a = S.a;
  const double r = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z)));
  if (r <= kCentreRel * a) {
    im.centre = true;
    im.x = 1e15 * a;
    im.y = im.z = 0.0;
    im.Q = 0.0;
    im.C = S.kc * q / a * (S.gam - 0.5 * S.dbar);
  } else {
    const double ar = __ddiv_rn(a, r);
    const double s = __dmul_rn(ar, ar);
    const double rK = __ddiv_rn(__dmul_rn(a, a), r);
    im.centre = false;
    im.x = __dmul_rn(s, x);
    im.y = __dmul_rn(s, y);
    im.z = __dmul_rn(s, z);
    im.Q = S.kc * (q / a * (S.gam * rK + S.dbar * (S.Rtau - rK) / 2.0));
    im.C = 0.0;
  }
  return im;
}

__device__ __forceinline__ double inv_dist64(double ax, double ay, double az, double bx, double by, double bz)
{
  const double dx = ax - bx, dy = ay - by, dz = az - bz;
  return 1.0 / sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));
}

__device__ __forceinline__ double img_pot(const Image& im, double x, double y, double z)
{
  return im.centre ? im.C : im.Q * inv_dist64(x, y, z, im.x, im.y, im.z);
}

// Surface kernels at point y (|y| = R_tau): G0 = 1/|x - y|; G1 is the dipole kernel of the
// path: FP32 path the dy -> 0 limit (R_tau - x.yhat)/d^3, FP64 path the central difference
// (1/d_- - 1/d_+)/dy = 2 (R_tau - x.yhat)/(d_+ d_- (d_+ + d_-)).
__device__ __forceinline__ void surf_kernels(const SysDev& S, double x, double y, double z, const dbl4& yl,
                                             double& g0, double& g1)
{
  const double dx = x - yl.x, dy = y - yl.y, dz = z - yl.z;
  const double d2 = dx * dx + dy * dy + dz * dz;
  g0 = rsqrt(d2);
  const double hx = yl.x * S.inv_Rt, hy = yl.y * S.inv_Rt, hz = yl.z * S.inv_Rt;  // |y| = R_tau
  const double xy = x * hx + y * hy + z * hz;
  if (S.prec == HSMA_FP64) {
    const double rm = S.Rtau - 0.5 * S.dy, rp = S.Rtau + 0.5 * S.dy;
    const double mx = x - rm * hx, my = y - rm * hy, mz = z - rm * hz;
    const double px = x - rp * hx, py = y - rp * hy, pz = z - rp * hz;
    const double dm = sqrt(mx * mx + my * my + mz * mz);
    const double dp = sqrt(px * px + py * py + pz * pz);
    g1 = 2.0 * (S.Rtau - xy) / (dp * dm * (dp + dm));
  } else {
    g1 = (S.Rtau - xy) * (g0 * g0 * g0);
  }
}

// Phi(y; A_x) and dPhi/dr for the coefficients of one charge q at x (addition theorem form).
__device__ __forceinline__ void charge_series(const SysDev& S, const double* __restrict__ Mn,
                                              const double* __restrict__ inv_np1, double x, double y, double z,
                                              double q, const dbl4& yl, double& phi, double& dphi)
{
  const double a = S.a;
  const double r2 = x * x + y * y + z * z;
  const double r = sqrt(r2);
  const double pref = S.kc_a * q;
  const double c = S.dbar * (S.Rt_a * r * S.inv_a - 1.0) * 0.5;
  if (r <= kCentreRel * a) {
    phi = pref * (Mn[S.mn] - S.gam - c);
    dphi = 0.0;
    return;
  }
  // |y| = R_tau on the auxiliary sphere
  const double t = (x * yl.x + y * yl.y + z * yl.z) * rsqrt(r2) * S.inv_Rt;
  const double u = r * S.Rt_a * S.inv_a;
  double P0 = 1.0, P1 = t, un = 1.0, s = 0.0, sd = 0.0;
  for (int n = 0; n <= S.p; ++n) {
    const double Pn = n == 0 ? P0 : P1;
    const double term = (Mn[S.mn + n] - S.gam - c) * un * Pn;
    s += term;
    sd += (double)n * term;
    if (n >= 1) {
      // Bonnet: (n+1) P_{n+1} = (2n+1) t P_n - n P_{n-1}
      const double Pn1 = ((2.0 * n + 1.0) * t * P1 - (double)n * P0) * inv_np1[n];
      P0 = P1;
      P1 = Pn1;
    }
    un *= u;
  }
  phi = pref * s;
  dphi = pref * sd * S.inv_Rt;
}

// The same series on the FP32 path, in double-float arithmetic (FP64 runs at ~1/73 of FP32 on
// this GPU, and the series is ~10 FP64 operations per order and point): per request the block
// prepares, for the new (side 0) and the old (side 1) position, a_n = k q/(eps1 a)
// (M_n - gamma - c) u^n and b_n = n a_n (u = r R_tau/a^2) and the unit vector xhat; per point
// the Legendre recurrence in t = xhat.yhat and the sums run in (hi, lo) pairs.
struct SeriesShared {
  df a[2][HSMA_P_MAX + 1];
  df b[2][HSMA_P_MAX + 1];
  double hat[2][3];
};

// All threads of the block call it (it ends with __syncthreads).
__device__ __forceinline__ void series_prepare(const SysDev& S, const double* __restrict__ Mn, double xn, double yn,
                                               double zn, double xo, double yo, double zo, double q,
                                               SeriesShared& sh)
{
  const int np = S.p + 1;
  const int t = threadIdx.x;
  if (t < 2 * np) {
    const int side = t / np, n = t - side * np;
    const double x = side ? xo : xn, y = side ? yo : yn, z = side ? zo : zn;
    const double r = sqrt(x * x + y * y + z * z);
    const bool centre = r <= kCentreRel * S.a;
    const double c = S.dbar * (S.Rt_a * r * S.inv_a - 1.0) * 0.5;
    const double u = r * S.Rt_a * S.inv_a;
    double un = 1.0, base = u;
    for (int e = n; e; e >>= 1) {  // u^n by squaring
      if (e & 1) un *= base;
      base *= base;
    }
    const double an = S.kc_a * q * (Mn[S.mn + n] - S.gam - c) * (centre ? (n == 0 ? 1.0 : 0.0) : un);
    sh.a[side][n] = df_from_double(an);
    sh.b[side][n] = df_from_double((double)n * an);
    if (n == 0) {
      const double inv = centre ? 0.0 : 1.0 / r;
      sh.hat[side][0] = x * inv;
      sh.hat[side][1] = y * inv;
      sh.hat[side][2] = z * inv;
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void series_eval(const SysDev& S, const SeriesShared& sh, int side, const dbl4& yl,
                                            const Tables& tab, double& phi, double& dphi)
{
  const double tc = (sh.hat[side][0] * yl.x + sh.hat[side][1] * yl.y + sh.hat[side][2] * yl.z) * S.inv_Rt;
  const df t = df_from_double(tc);
  df P0 = df_make(1.f, 0.f), P1 = t;
  df s = sh.a[side][0], sd = df_make(0.f, 0.f);
  for (int n = 1; n <= S.p; ++n) {
    s = df_acc(s, sh.a[side][n], P1);
    sd = df_acc(sd, sh.b[side][n], P1);
    if (n < S.p) {
      const float2 la = tab.leg_a2[n], lb = tab.leg_b2[n];
      const df A = df_make(la.x, la.y) * t;
      const df P2 = df_mul_sub(A, P1, df_make(lb.x, lb.y), P0);
      P0 = P1;
      P1 = P2;
    }
  }
  phi = df_to_double(df_norm(s));
  dphi = df_to_double(df_norm(sd)) * S.inv_Rt;
}

// Work item: (request, kind 0 = rows / 1 = surface, block)
__global__ __launch_bounds__(kDeltaThreads) void k_delta(const SysDev* __restrict__ sys, const int4* __restrict__ items,
                                                         int nitems, const int2* __restrict__ req_items,
                                                         const DeltaReq* __restrict__ reqs, int nreq,
                                                         const double* __restrict__ xyz, const double* __restrict__ q,
                                                         const int* __restrict__ perm, const int* __restrict__ iperm,
                                                         const float4* __restrict__ src_hi,
                                                         const float4* __restrict__ src_lo,
                                                         const dbl4* __restrict__ src64, const dbl4* __restrict__ surfx,
                                                         const double2* __restrict__ surfqd,
                                                         const double2* __restrict__ vsurf,
                                                         const double* __restrict__ Mn, Tables tab,
                                                         double* __restrict__ dpart, double* __restrict__ de,
                                                         unsigned int* __restrict__ counter, int* __restrict__ status)
{
  __shared__ double red[kDeltaThreads / 32];
  __shared__ bool last;
  __shared__ SeriesShared ssh;
  __shared__ Image s_in, s_io;
  const double* inv_np1 = tab.inv_np1;
  const int4 it = items[blockIdx.x];
  const DeltaReq R = reqs[it.x];
  const SysDev& S = sys[R.sys];
  const long long kk = S.chg + R.k;
  const double xo = xyz[3 * kk], yo = xyz[3 * kk + 1], zo = xyz[3 * kk + 2], qk = q[kk];
  const double xn = R.x, yn = R.y, zn = R.z;
  double acc = 0.0;
  const int idx = it.z * kDeltaThreads + threadIdx.x;
  if (it.y == 0) {
    // the moved charge's images (FP64), once per block
    if (threadIdx.x == 0) {
      s_in = kelvin_image(S, xn, yn, zn, qk);
      s_io = kelvin_image(S, xo, yo, zo, qk);
    }
    __syncthreads();
    const Image In = s_in, Io = s_io;
    if (blockIdx.x == req_items[it.x].x && threadIdx.x == 0) {
      const double rn2 = xn * xn + yn * yn + zn * zn;
      if (!(rn2 < S.a * S.a) || !isfinite(rn2)) atomicOr(status, kStBadMove);
      // the moved charge and its own image
      acc += 0.5 * qk * (img_pot(In, xn, yn, zn) - img_pot(Io, xo, yo, zo));
    }
    // rows run over sorted positions j (records are in the spatial order of k_order.cu)
    const int j = idx;
    if (j < S.n && j != iperm[kk]) {
      const double qj = q[S.chg + perm[S.chg + j]];
      if (S.prec == HSMA_FP64) {
        const dbl4 rj = src64[S.src + j];
        const dbl4 kj = src64[S.src + S.n + j];
        const double cn = inv_dist64(xn, yn, zn, rj.x, rj.y, rj.z), co = inv_dist64(xo, yo, zo, rj.x, rj.y, rj.z);
        acc += qk * rj.w * (cn - co);
        if (kj.w != 0.0) acc += 0.5 * qk * kj.w * (inv_dist64(xn, yn, zn, kj.x, kj.y, kj.z) -
                                                   inv_dist64(xo, yo, zo, kj.x, kj.y, kj.z));
        acc += 0.5 * qj * (img_pot(In, rj.x, rj.y, rj.z) - img_pot(Io, rj.x, rj.y, rj.z));
      } else {
        float nh[3], nl[3], oh[3], ol[3];
        split_hilo(xn, nh[0], nl[0]); split_hilo(yn, nh[1], nl[1]); split_hilo(zn, nh[2], nl[2]);
        split_hilo(xo, oh[0], ol[0]); split_hilo(yo, oh[1], ol[1]); split_hilo(zo, oh[2], ol[2]);
        const float4 rh = src_hi[S.src + j], rl = src_lo[S.src + j];
        const float4 kh = src_hi[S.src + S.n + j], kl = src_lo[S.src + S.n + j];
        float t = rh.w * (inv_hilo(nh[0], nh[1], nh[2], nl[0], nl[1], nl[2], rh.x, rh.y, rh.z, rl.x, rl.y, rl.z) -
                          inv_hilo(oh[0], oh[1], oh[2], ol[0], ol[1], ol[2], rh.x, rh.y, rh.z, rl.x, rl.y, rl.z));
        acc += qk * (double)t;
        t = kh.w * (inv_hilo(nh[0], nh[1], nh[2], nl[0], nl[1], nl[2], kh.x, kh.y, kh.z, kl.x, kl.y, kl.z) -
                    inv_hilo(oh[0], oh[1], oh[2], ol[0], ol[1], ol[2], kh.x, kh.y, kh.z, kl.x, kl.y, kl.z));
        acc += 0.5 * qk * (double)t;
        // j's charge in k's image potential (images split hi/lo like the records)
        float ih[3], il[3], jh[3], jl[3];
        double pn, po;
        if (In.centre) {
          pn = In.C;
        } else {
          split_hilo(In.x, ih[0], il[0]); split_hilo(In.y, ih[1], il[1]); split_hilo(In.z, ih[2], il[2]);
          jh[0] = rh.x; jh[1] = rh.y; jh[2] = rh.z; jl[0] = rl.x; jl[1] = rl.y; jl[2] = rl.z;
          pn = In.Q * (double)inv_hilo(jh[0], jh[1], jh[2], jl[0], jl[1], jl[2], ih[0], ih[1], ih[2], il[0], il[1], il[2]);
        }
        if (Io.centre) {
          po = Io.C;
        } else {
          split_hilo(Io.x, ih[0], il[0]); split_hilo(Io.y, ih[1], il[1]); split_hilo(Io.z, ih[2], il[2]);
          po = Io.Q * (double)inv_hilo(rh.x, rh.y, rh.z, rl.x, rl.y, rl.z, ih[0], ih[1], ih[2], il[0], il[1], il[2]);
        }
        acc += 0.5 * qj * (pn - po);
      }
    }
  } else {
    const bool dfs = S.prec != HSMA_FP64;
    if (dfs) series_prepare(S, Mn, xn, yn, zn, xo, yo, zo, qk, ssh);
    const int l = idx;
    if (l < S.M) {
      const dbl4 yl = surfx[S.surf + l];
      const double2 QD = surfqd[S.surf + l];
      const double2 V = vsurf[S.surf + l];
      double g0n, g1n, g0o, g1o, pn, dpn, po, dpo;
      surf_kernels(S, xn, yn, zn, yl, g0n, g1n);
      surf_kernels(S, xo, yo, zo, yl, g0o, g1o);
      if (dfs) {
        series_eval(S, ssh, 0, yl, tab, pn, dpn);
        series_eval(S, ssh, 1, yl, tab, po, dpo);
      } else {
        charge_series(S, Mn, inv_np1, xn, yn, zn, qk, yl, pn, dpn);
        charge_series(S, Mn, inv_np1, xo, yo, zo, qk, yl, po, dpo);
      }
      const double w4 = yl.w / (4.0 * kPi);
      const double dQ0 = w4 * (dpn - dpo), dD = w4 * (pn - po);
      const double dV0 = qk * (g0n - g0o), dV1 = qk * (g1n - g1o);
      acc += 0.5 * (dQ0 * (V.x + dV0) + QD.x * dV0 + dD * (V.y + dV1) + QD.y * dV1);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kDeltaThreads / 32; ++w) s += red[w];
    dpart[blockIdx.x] = s;
    __threadfence();
    last = atomicAdd(counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int r = threadIdx.x; r < nreq; r += kDeltaThreads) {
    const int2 rg = req_items[r];
    double s = 0.0;
    for (int i = 0; i < rg.y; ++i) s += ((volatile double*)dpart)[rg.x + i];
    de[r] = s;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// Potentials of the real charges under the two surface kernels, V0_l and V1_l (FP64; one warp
// per surface point, fixed lane order and shuffle tree).
__global__ __launch_bounds__(256) void k_surface_potentials(const SysDev* __restrict__ sys,
                                                            const int2* __restrict__ items,
                                                            const double* __restrict__ xyz,
                                                            const double* __restrict__ q,
                                                            const dbl4* __restrict__ surfx, double2* __restrict__ vsurf)
{
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int l = it.y * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (l >= S.M) return;
  const dbl4 yl = surfx[S.surf + l];
  double v0 = 0.0, v1 = 0.0;
  for (int i = lane; i < S.n; i += 32) {
    const long long g = S.chg + i;
    double g0, g1;
    surf_kernels(S, xyz[3 * g], xyz[3 * g + 1], xyz[3 * g + 2], yl, g0, g1);
    v0 += q[g] * g0;
    v1 += q[g] * g1;
  }
  for (int o = 16; o > 0; o >>= 1) {
    v0 += __shfl_xor_sync(0xffffffffu, v0, o);
    v1 += __shfl_xor_sync(0xffffffffu, v1, o);
  }
  if (lane == 0) vsurf[S.surf + l] = make_double2(v0, v1);
}

// Order-independent float min/max in global memory (integer atomics on the bit patterns:
// signed for non-negative values, unsigned for values with the sign bit set), so boxes
// grown by several moves of one launch do not depend on their order.
__device__ __forceinline__ void atomic_min_f(float* a, float v)
{
  if (!signbit(v))
    atomicMin(reinterpret_cast<int*>(a), __float_as_int(v));
  else
    atomicMax(reinterpret_cast<unsigned int*>(a), __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_f(float* a, float v)
{
  if (!signbit(v))
    atomicMax(reinterpret_cast<int*>(a), __float_as_int(v));
  else
    atomicMin(reinterpret_cast<unsigned int*>(a), __float_as_uint(v));
}
// box = (min, max) float4 pair: grow it to contain (x, y, z)
__device__ __forceinline__ void box_grow(float4* box, float x, float y, float z)
{
  atomic_min_f(&box[0].x, x);
  atomic_min_f(&box[0].y, y);
  atomic_min_f(&box[0].z, z);
  atomic_max_f(&box[1].x, x);
  atomic_max_f(&box[1].y, y);
  atomic_max_f(&box[1].z, z);
}

// Commit of a move, surface part: Q0, D, V0, V1 and the pair-sum surface records of every point.
// Must run before k_move_charge (it reads the old position).
__global__ __launch_bounds__(256) void k_move_surface(const SysDev* __restrict__ sys, const int2* __restrict__ items,
                                                      const DeltaReq* __restrict__ reqs, const double* __restrict__ xyz,
                                                      const double* __restrict__ q, const double* __restrict__ Mn,
                                                      Tables tab, const dbl4* __restrict__ surfx,
                                                      double2* __restrict__ surfqd,
                                                      double2* __restrict__ vsurf, int have_v,
                                                      float4* __restrict__ surf_a, float4* __restrict__ surf_b,
                                                      dbl4* __restrict__ surf64_a, double* __restrict__ surf64_b)
{
  __shared__ SeriesShared ssh;
  const int2 it = items[blockIdx.x];  // (request, block)
  const DeltaReq R = reqs[it.x];
  const SysDev& S = sys[R.sys];
  const long long kk = S.chg + R.k;
  const double xo = xyz[3 * kk], yo = xyz[3 * kk + 1], zo = xyz[3 * kk + 2], qk = q[kk];
  const bool dfs = S.prec != HSMA_FP64;
  if (dfs) series_prepare(S, Mn, R.x, R.y, R.z, xo, yo, zo, qk, ssh);
  const int l = it.y * 256 + threadIdx.x;
  if (l >= S.M) return;
  const long long o = S.surf + l;
  const dbl4 yl = surfx[o];
  double pn, dpn, po, dpo;
  if (dfs) {
    series_eval(S, ssh, 0, yl, tab, pn, dpn);
    series_eval(S, ssh, 1, yl, tab, po, dpo);
  } else {
    charge_series(S, Mn, tab.inv_np1, R.x, R.y, R.z, qk, yl, pn, dpn);
    charge_series(S, Mn, tab.inv_np1, xo, yo, zo, qk, yl, po, dpo);
  }
  const double w4 = yl.w / (4.0 * kPi);
  double2 QD = surfqd[o];
  QD.x += w4 * (dpn - dpo);
  QD.y += w4 * (pn - po);
  surfqd[o] = QD;
  if (have_v) {
    double g0n, g1n, g0o, g1o;
    surf_kernels(S, R.x, R.y, R.z, yl, g0n, g1n);
    surf_kernels(S, xo, yo, zo, yl, g0o, g1o);
    double2 V = vsurf[o];
    V.x += qk * (g0n - g0o);
    V.y += qk * (g1n - g1o);
    vsurf[o] = V;
  }
  if (S.prec == HSMA_FP64) {
    surf64_a[o] = make_dbl4(yl.x, yl.y, yl.z, QD.x);
    surf64_b[o] = QD.y;
  } else {
    surf_a[o] = make_float4((float)yl.x, (float)yl.y, (float)yl.z, (float)QD.x);
    surf_b[o] = make_float4((float)(-QD.y / S.Rtau), 0.f, 0.f, 0.f);
  }
}

// Commit of a move, charge part (one block per request): coefficients A += dA (two solid-harmonic
// columns sets computed by warps 0 and 1), the real and Kelvin records of k, the centre constant,
// and the position itself.
__global__ __launch_bounds__(256) void k_move_charge(const SysDev* __restrict__ sys, const DeltaReq* __restrict__ reqs,
                                                     Tables tab, double* __restrict__ xyz, const double* __restrict__ q,
                                                     const double* __restrict__ Mn, double* __restrict__ coef,
                                                     float2* __restrict__ coef2, double* __restrict__ r0,
                                                     const int* __restrict__ iperm, float4* __restrict__ src_hi,
                                                     float4* __restrict__ src_lo, dbl4* __restrict__ src64,
                                                     float4* __restrict__ boxes)
{
  extern __shared__ double sm[];
  const DeltaReq R = reqs[blockIdx.x];
  const SysDev& S = sys[R.sys];
  const int P = S.P, p = S.p;
  double* Tn = sm;
  double* To = sm + P;
  const long long kk = S.chg + R.k;
  const double xo = xyz[3 * kk], yo = xyz[3 * kk + 1], zo = xyz[3 * kk + 2], qk = q[kk];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const double a = S.a;
  if (warp < 2) {
    const double x = (warp == 0 ? R.x : xo) / a, y = (warp == 0 ? R.y : yo) / a, z = (warp == 0 ? R.z : zo) / a;
    const double rho2 = x * x + y * y + z * z;
    double* T = warp == 0 ? Tn : To;
    for (int m = lane; m <= p; m += 32) {
      double cr = 1.0, ci = 0.0;
      for (int kq = 1; kq <= m; ++kq) {
        const double f = tab.sect[kq];
        const double nr = f * (cr * x - ci * y);
        const double ni = f * (cr * y + ci * x);
        cr = nr;
        ci = ni;
      }
      T[m * m + m + m] = cr;
      if (m) T[m * m + m - m] = ci;
      double pr = cr, pi = ci, qr = 0.0, qi = 0.0;
      for (int n = m + 1; n <= p; ++n) {
        const int t = n * (n + 1) / 2 + m;
        const double A = tab.rec_a[t] * z, B = tab.rec_b[t] * rho2;
        const double nr = A * pr - B * qr;
        const double ni = A * pi - B * qi;
        T[n * n + n + m] = nr;
        if (m) T[n * n + n - m] = ni;
        qr = pr;
        qi = pi;
        pr = nr;
        pi = ni;
      }
    }
  }
  __syncthreads();
  const double rn = sqrt(R.x * R.x + R.y * R.y + R.z * R.z), ro = sqrt(xo * xo + yo * yo + zo * zo);
  const double cn = S.dbar * (S.Rtau * rn / (a * a) - 1.0) * 0.5;
  const double co = S.dbar * (S.Rtau * ro / (a * a) - 1.0) * 0.5;
  for (int idx = threadIdx.x; idx < P; idx += blockDim.x) {
    int n = (int)sqrt((double)idx);
    while (n * n > idx) --n;
    while ((n + 1) * (n + 1) <= idx) ++n;
    const double mg = Mn[S.mn + n] - S.gam;
    const double c = coef[S.coef + idx] + S.kc / a * qk * ((mg - cn) * Tn[idx] - (mg - co) * To[idx]);
    coef[S.coef + idx] = c;
    float ch, cl;
    split_double(c, ch, cl);
    coef2[S.coef + idx] = make_float2(ch, cl);
  }
  if (threadIdx.x == 0) {
    const Image In = kelvin_image(S, R.x, R.y, R.z, qk);
    const Image Io = kelvin_image(S, xo, yo, zo, qk);
    r0[R.sys] += In.C - Io.C;
    // the records sit at k's sorted position; its boxes grow to cover the new points (the
    // order itself is refreshed by the next full build)
    const int ks = iperm[kk];
    const long long sr = S.src + ks, sk = S.src + S.n + ks;
    if (S.prec == HSMA_FP64) {
      src64[sr] = make_dbl4(R.x, R.y, R.z, S.kc * qk);
      src64[sk] = make_dbl4(In.x, In.y, In.z, In.Q);
    } else {
      float hx, hy, hz, lx, ly, lz;
      // (the lo records' fourth components: the weights of the symmetric pair sum's transposed
      // Kelvin term, as written by k_images)
      const double rn2 = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(R.x, R.x), __dmul_rn(R.y, R.y)), __dmul_rn(R.z, R.z)));
      split_hilo(R.x, hx, lx); split_hilo(R.y, hy, ly); split_hilo(R.z, hz, lz);
      src_hi[sr] = make_float4(hx, hy, hz, (float)(S.kc * qk));
      src_lo[sr] = make_float4(lx, ly, lz, In.centre ? 0.f : (float)(In.Q * rn2));
      const long long b = S.bb + ks / kBox, bk = b + (S.n + kBox - 1) / kBox;
      box_grow(boxes + 2 * b, hx, hy, hz);
      split_hilo(In.x, hx, lx); split_hilo(In.y, hy, ly); split_hilo(In.z, hz, lz);
      src_hi[sk] = make_float4(hx, hy, hz, (float)In.Q);
      src_lo[sk] = make_float4(lx, ly, lz, In.centre ? (float)(1e15 * S.inv_a) : (float)(1.0 / rn2));
      if (!In.centre) box_grow(boxes + 2 * bk, hx, hy, hz);
    }
    xyz[3 * kk] = R.x;
    xyz[3 * kk + 1] = R.y;
    xyz[3 * kk + 2] = R.z;
  }
}

// ---------------------------------------------------------------------------------------
void launch_surface_potentials(const SysDev* sys, const int2* items, int nitems, const double* xyz, const double* q,
                               const dbl4* surfx, double2* vsurf, cudaStream_t st)
{
  if (nitems <= 0) return;
  k_surface_potentials<<<nitems, 256, 0, st>>>(sys, items, xyz, q, surfx, vsurf);
}

void launch_delta(const SysDev* sys, const int4* items, int nitems, const int2* req_items, const DeltaReq* reqs,
                  int nreq, const double* xyz, const double* q, const int* perm, const int* iperm,
                  const float4* src_hi, const float4* src_lo, const dbl4* src64, const dbl4* surfx,
                  const double2* surfqd, const double2* vsurf, const double* Mn, Tables tab, double* dpart,
                  double* de, unsigned int* counter, int* status, cudaStream_t st)
{
  if (nitems <= 0) return;
  k_delta<<<nitems, kDeltaThreads, 0, st>>>(sys, items, nitems, req_items, reqs, nreq, xyz, q, perm, iperm, src_hi,
                                            src_lo, src64, surfx, surfqd, vsurf, Mn, tab, dpart, de, counter, status);
}

void launch_move(const SysDev* sys, const int2* surf_items, int n_surf_items, const DeltaReq* reqs, int nreq,
                 Tables tab, int maxP, double* xyz, const double* q, const double* Mn, double* coef, float2* coef2,
                 double* r0, const dbl4* surfx, double2* surfqd, double2* vsurf, int have_v, float4* surf_a,
                 float4* surf_b, dbl4* surf64_a, double* surf64_b, const int* iperm, float4* src_hi, float4* src_lo,
                 dbl4* src64, float4* boxes, cudaStream_t st)
{
  if (nreq <= 0) return;
  if (n_surf_items > 0)
    k_move_surface<<<n_surf_items, 256, 0, st>>>(sys, surf_items, reqs, xyz, q, Mn, tab, surfx, surfqd,
                                                 vsurf, have_v, surf_a, surf_b, surf64_a, surf64_b);
  k_move_charge<<<nreq, 256, 2 * (size_t)maxP * sizeof(double), st>>>(sys, reqs, tab, xyz, q, Mn,
                                                                     coef, coef2, r0, iperm, src_hi, src_lo, src64,
                                                                     boxes);
}

void init_delta_kernels()
{
  cudaFuncSetAttribute(k_move_charge, cudaFuncAttributeMaxDynamicSharedMemorySize, 120 * 1024);
}

}  // namespace hsma
