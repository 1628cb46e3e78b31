// Fields E = -grad phi at every charge, together with the potential, in one pass over the same
// source set as k_pairs.cu (real charges except the target itself, Kelvin images, the monopole
// and dipole layers of the auxiliary sphere; Sec. 2.4, eqs. phicorrfinall and phirffinall),
// differentiated term by term with the sources fixed, so that F_i = q_i E(x_i).
//
// Work items, chunking, spatial order and the near/far box test are those of the potential
// pass.  Per (chunk, target) the FP32 kernel writes two float4, the (hi, lo) two-sum pairs of
// (phi, Ex, Ey, Ez); the FP64 kernel one (phi, Ex, Ey, Ez) in double.  k_reduce_field sums
// them in a fixed order (double-float on the FP32 path) and maps them back to input order.
//   point source Q at s:   phi += Q/d,  E += Q (t - s)/d^3
//   surface point y (FP32, the dy -> 0 limit of the dipole pair, Dp = -D/R_tau):
//     phi += (Q0 + Dp u)/d,  u = ((t - y).y)/d^2,
//     E   += [(Q0 + 3 Dp u)(t - y) - Dp y] / d^3
//   surface point y (FP64, the central difference itself, written without cancellation):
//     E += Q0 (t - y)/d^3 + D [ yhat/d_-^3 + (t - y^+) 2 (R_tau - t.yhat)(d_+^2 + d_+ d_- + d_-^2)
//                                           / ((d_+ + d_-) d_-^3 d_+^3) ]
#include <math.h>

#include "df64.cuh"
#include "fp32_pair.cuh"
#include "hsma_internal.cuh"

namespace hsma {


struct FChunk {
  int type;       // 0 real, 1 Kelvin, 2 surface
  int first;      // index of the first source within its kind
  int count;
  long long off;  // record offset of the first source
};

__device__ __forceinline__ FChunk field_chunk(const SysDev& S, int c)
{
  FChunk ci;
  if (c < S.ncr) {
    ci.type = 0;
    ci.first = c * S.chunk;
    ci.count = min(S.chunk, S.n - ci.first);
    ci.off = S.src + ci.first;
  } else if (c < S.ncr + S.nck) {
    ci.type = 1;
    ci.first = (c - S.ncr) * S.chunk;
    ci.count = min(S.chunk, S.n - ci.first);
    ci.off = S.src + S.n + ci.first;
  } else {
    ci.type = 2;
    ci.first = (c - S.ncr - S.nck) * S.chunk_s;
    ci.count = min(S.chunk_s, S.M - ci.first);
    ci.off = S.surf + ci.first;
  }
  return ci;
}

// a += b as an (hi, lo) two-sum fold
__device__ __forceinline__ void fold(float& H, float& L, float b)
{
  const float s = H + b;
  const float bp = s - H;
  L += (H - (s - bp)) + (b - bp);
  H = s;
}

template <int NT, int K>
__global__ __launch_bounds__(NT) void k_field_f32(const SysDev* __restrict__ sys, PairWork w1, PairWork w2,
                                                  const float4* __restrict__ src_hi,
                                                  const float4* __restrict__ src_lo,
                                                  const float4* __restrict__ surf_a,
                                                  const float4* __restrict__ surf_b,
                                                  const float4* __restrict__ boxes, float4* __restrict__ fpart)
{
  static_assert(NT % kBox == 0, "a staged tile holds whole source boxes");
  __shared__ __align__(16) float4 shA[2][NT];
  __shared__ __align__(16) float4 shB[2][NT];
  __shared__ int s_item, s_list;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int list = 0;
  bool first_fetch = true;
  grid_dependency_wait();  // (a programmatic launch: the records and counters of the pass)

  for (;;) {
    if (tid == 0) next_pair_item(w1, w2, list, first_fetch, s_item, s_list);
    first_fetch = false;
    __syncthreads();
    const int item = s_item;
    list = s_list;
    __syncthreads();
    if (list > 1) break;
    const int4 it = (list == 0 ? w1.items : w2.items)[item];
    const SysDev& S = sys[it.x];
    const int n = S.n;
    const int t0 = it.y * (NT * K);
    const int w0 = t0 + warp * 32 * K;
    const FChunk ch = field_chunk(S, it.z);

    // the first source tile is in flight while the targets load
    const float4* gA = ch.type == 2 ? surf_a + ch.off : src_hi + ch.off;
    const float4* gB = ch.type == 2 ? surf_b + ch.off : src_lo + ch.off;
    const int ntiles = (ch.count + NT - 1) / NT;
    const long long box_kind = S.bb + (ch.type == 1 ? (n + kBox - 1) / kBox : 0);

    if (tid < ch.count) {
      cp_async16(&shA[0][tid], gA + tid);
      cp_async16(&shB[0][tid], gB + tid);
    }
    cp_async_commit();

    float txh[K], tyh[K], tzh[K], txl[K], tyl[K], tzl[K];
    int tix[K];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const int i = w0 + k * 32 + lane;
      const int ii = i < n ? i : t0;
      tix[k] = i;
      const float4 h = src_hi[S.src + ii];
      const float4 l = src_lo[S.src + ii];
      txh[k] = h.x; tyh[k] = h.y; tzh[k] = h.z;
      txl[k] = l.x; tyl[k] = l.y; tzl[k] = l.z;
    }
    float wmnx = txh[0], wmny = tyh[0], wmnz = tzh[0], wmxx = txh[0], wmxy = tyh[0], wmxz = tzh[0];
#pragma unroll
    for (int k = 1; k < K; ++k) {
      wmnx = fminf(wmnx, txh[k]); wmny = fminf(wmny, tyh[k]); wmnz = fminf(wmnz, tzh[k]);
      wmxx = fmaxf(wmxx, txh[k]); wmxy = fmaxf(wmxy, tyh[k]); wmxz = fmaxf(wmxz, tzh[k]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      wmnx = fminf(wmnx, __shfl_xor_sync(0xffffffffu, wmnx, o));
      wmny = fminf(wmny, __shfl_xor_sync(0xffffffffu, wmny, o));
      wmnz = fminf(wmnz, __shfl_xor_sync(0xffffffffu, wmnz, o));
      wmxx = fmaxf(wmxx, __shfl_xor_sync(0xffffffffu, wmxx, o));
      wmxy = fmaxf(wmxy, __shfl_xor_sync(0xffffffffu, wmxy, o));
      wmxz = fmaxf(wmxz, __shfl_xor_sync(0xffffffffu, wmxz, o));
    }
    float Hp[K], Lp[K], Hx[K], Lx[K], Hy[K], Ly[K], Hz[K], Lz[K];
#pragma unroll
    for (int k = 0; k < K; ++k) Hp[k] = Lp[k] = Hx[k] = Lx[k] = Hy[k] = Ly[k] = Hz[k] = Lz[k] = 0.f;

    for (int t = 0; t < ntiles; ++t) {
      const int buf = t & 1;
      if (t + 1 < ntiles) {
        const int s = (t + 1) * NT + tid;
        if (s < ch.count) {
          cp_async16(&shA[buf ^ 1][tid], gA + s);
          cp_async16(&shB[buf ^ 1][tid], gB + s);
        }
        cp_async_commit();
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();
      const int cnt = min(NT, ch.count - t * NT);
      const float4* A = shA[buf];
      const float4* B = shB[buf];
      float ap[K], ax[K], ay[K], az[K];
#pragma unroll
      for (int k = 0; k < K; ++k) ap[k] = ax[k] = ay[k] = az[k] = 0.f;
      if (ch.type == 2 && K % 2 == 0) {
        // packed FP32 over target slots 2h, 2h + 1 (FFMA2 / FADD2 / FMUL2, each component
        // rounded as the scalar form below: the same sums, half the FP32 issue slots)
        constexpr int H = K / 2 > 0 ? K / 2 : 1;
        float2 X[H], Y[H], Z[H], AP[H], AX[H], AY[H], AZ[H];
#pragma unroll
        for (int h = 0; h < K / 2; ++h) {
          X[h] = make_float2(txh[2 * h], txh[2 * h + 1]);
          Y[h] = make_float2(tyh[2 * h], tyh[2 * h + 1]);
          Z[h] = make_float2(tzh[2 * h], tzh[2 * h + 1]);
          AP[h] = AX[h] = AY[h] = AZ[h] = make_float2(0.f, 0.f);
        }
        for (int s = 0; s < cnt; ++s) {
          const float4 y = A[s];
          const float Dp = B[s].x;
          const float Dp3 = 3.f * Dp;
          const float2 yx = make_float2(y.x, y.x), yy = make_float2(y.y, y.y), yz = make_float2(y.z, y.z);
          const float2 yw = make_float2(y.w, y.w), dp = make_float2(Dp, Dp), dp3 = make_float2(Dp3, Dp3);
          const float2 ndp = make_float2(-Dp, -Dp);
#pragma unroll
          for (int h = 0; h < K / 2; ++h) {
            const float2 dx = __fadd2_rn(X[h], make_float2(-y.x, -y.x));
            const float2 dy = __fadd2_rn(Y[h], make_float2(-y.y, -y.y));
            const float2 dz = __fadd2_rn(Z[h], make_float2(-y.z, -y.z));
            float2 r2 = __fmul2_rn(dx, dx);
            r2 = __ffma2_rn(dy, dy, r2);
            r2 = __ffma2_rn(dz, dz, r2);
            const float2 inv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
            const float2 inv2 = __fmul2_rn(inv, inv);
            float2 dot = __fmul2_rn(dx, yx);
            dot = __ffma2_rn(dy, yy, dot);
            dot = __ffma2_rn(dz, yz, dot);
            const float2 u = __fmul2_rn(dot, inv2);
            AP[h] = __ffma2_rn(__ffma2_rn(dp, u, yw), inv, AP[h]);
            const float2 inv3 = __fmul2_rn(inv, inv2);
            const float2 c0 = __fmul2_rn(__ffma2_rn(dp3, u, yw), inv3);
            const float2 c1 = __fmul2_rn(ndp, inv3);
            AX[h] = __ffma2_rn(c1, yx, __ffma2_rn(c0, dx, AX[h]));
            AY[h] = __ffma2_rn(c1, yy, __ffma2_rn(c0, dy, AY[h]));
            AZ[h] = __ffma2_rn(c1, yz, __ffma2_rn(c0, dz, AZ[h]));
          }
        }
#pragma unroll
        for (int h = 0; h < K / 2; ++h) {
          ap[2 * h] = AP[h].x; ap[2 * h + 1] = AP[h].y;
          ax[2 * h] = AX[h].x; ax[2 * h + 1] = AX[h].y;
          ay[2 * h] = AY[h].x; ay[2 * h + 1] = AY[h].y;
          az[2 * h] = AZ[h].x; az[2 * h + 1] = AZ[h].y;
        }
      } else if (ch.type == 2) {
        for (int s = 0; s < cnt; ++s) {
          const float4 y = A[s];
          const float Dp = B[s].x;
          const float Dp3 = 3.f * Dp;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const float dx = txh[k] - y.x, dy = tyh[k] - y.y, dz = tzh[k] - y.z;
            float r2 = dx * dx;
            r2 = fmaf(dy, dy, r2);
            r2 = fmaf(dz, dz, r2);
            const float inv = rsqrt_mufu(r2);
            const float inv2 = inv * inv;
            float dot = dx * y.x;
            dot = fmaf(dy, y.y, dot);
            dot = fmaf(dz, y.z, dot);
            const float u = dot * inv2;
            ap[k] = fmaf(fmaf(Dp, u, y.w), inv, ap[k]);
            const float inv3 = inv * inv2;
            const float c0 = fmaf(Dp3, u, y.w) * inv3;
            const float c1 = -Dp * inv3;
            ax[k] = fmaf(c1, y.x, fmaf(c0, dx, ax[k]));
            ay[k] = fmaf(c1, y.y, fmaf(c0, dy, ay[k]));
            az[k] = fmaf(c1, y.z, fmaf(c0, dz, az[k]));
          }
        }
      } else {
        const int sbase = ch.first + t * NT;
        for (int u = 0; u < cnt; u += kBox) {
          const int ue = min(cnt, u + kBox);
          const long long bi = box_kind + (sbase + u) / kBox;
          const float4 bmn = __ldg(&boxes[2 * bi]), bmx = __ldg(&boxes[2 * bi + 1]);
          const float gx = fmaxf(0.f, fmaxf(wmnx - bmx.x, bmn.x - wmxx));
          const float gy = fmaxf(0.f, fmaxf(wmny - bmx.y, bmn.y - wmxy));
          const float gz = fmaxf(0.f, fmaxf(wmnz - bmx.z, bmn.z - wmxz));
          if (gx * gx + gy * gy + gz * gz > S.dc2 && K % 2 == 0) {
            // packed, as the surface sums above
            constexpr int H = K / 2 > 0 ? K / 2 : 1;
            float2 X[H], Y[H], Z[H], AP[H], AX[H], AY[H], AZ[H];
#pragma unroll
            for (int h = 0; h < K / 2; ++h) {
              X[h] = make_float2(txh[2 * h], txh[2 * h + 1]);
              Y[h] = make_float2(tyh[2 * h], tyh[2 * h + 1]);
              Z[h] = make_float2(tzh[2 * h], tzh[2 * h + 1]);
              AP[h] = make_float2(ap[2 * h], ap[2 * h + 1]);
              AX[h] = make_float2(ax[2 * h], ax[2 * h + 1]);
              AY[h] = make_float2(ay[2 * h], ay[2 * h + 1]);
              AZ[h] = make_float2(az[2 * h], az[2 * h + 1]);
            }
#pragma unroll 2
            for (int s = u; s < ue; ++s) {
              const float4 hs = A[s];
              const float2 hw = make_float2(hs.w, hs.w);
#pragma unroll
              for (int h = 0; h < K / 2; ++h) {
                const float2 dx = __fadd2_rn(X[h], make_float2(-hs.x, -hs.x));
                const float2 dy = __fadd2_rn(Y[h], make_float2(-hs.y, -hs.y));
                const float2 dz = __fadd2_rn(Z[h], make_float2(-hs.z, -hs.z));
                float2 r2 = __fmul2_rn(dx, dx);
                r2 = __ffma2_rn(dy, dy, r2);
                r2 = __ffma2_rn(dz, dz, r2);
                const float2 inv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
                const float2 qi = __fmul2_rn(hw, inv);
                AP[h] = __fadd2_rn(AP[h], qi);
                const float2 c = __fmul2_rn(qi, __fmul2_rn(inv, inv));
                AX[h] = __ffma2_rn(c, dx, AX[h]);
                AY[h] = __ffma2_rn(c, dy, AY[h]);
                AZ[h] = __ffma2_rn(c, dz, AZ[h]);
              }
            }
#pragma unroll
            for (int h = 0; h < K / 2; ++h) {
              ap[2 * h] = AP[h].x; ap[2 * h + 1] = AP[h].y;
              ax[2 * h] = AX[h].x; ax[2 * h + 1] = AX[h].y;
              ay[2 * h] = AY[h].x; ay[2 * h + 1] = AY[h].y;
              az[2 * h] = AZ[h].x; az[2 * h + 1] = AZ[h].y;
            }
          } else if (gx * gx + gy * gy + gz * gz > S.dc2) {
#pragma unroll 2
            for (int s = u; s < ue; ++s) {
              const float4 h = A[s];
#pragma unroll
              for (int k = 0; k < K; ++k) {
                const float dx = txh[k] - h.x, dy = tyh[k] - h.y, dz = tzh[k] - h.z;
                float r2 = dx * dx;
                r2 = fmaf(dy, dy, r2);
                r2 = fmaf(dz, dz, r2);
                const float inv = rsqrt_mufu(r2);
                const float qi = h.w * inv;
                ap[k] += qi;
                const float c = qi * (inv * inv);
                ax[k] = fmaf(c, dx, ax[k]);
                ay[k] = fmaf(c, dy, ay[k]);
                az[k] = fmaf(c, dz, az[k]);
              }
            }
          } else {
            const bool self = ch.type == 0 && sbase + u < w0 + 32 * K && w0 < sbase + ue;
            for (int s = u; s < ue; ++s) {
              const float4 h = A[s];
              const float4 l = B[s];
#pragma unroll
              for (int k = 0; k < K; ++k) {
                const float dx = txh[k] - h.x, dy = tyh[k] - h.y, dz = tzh[k] - h.z;
                const float ex = (txl[k] - l.x) + dx, ey = (tyl[k] - l.y) + dy, ez = (tzl[k] - l.z) + dz;
                float r2 = ex * ex;
                r2 = fmaf(ey, ey, r2);
                r2 = fmaf(ez, ez, r2);
                float inv = rsqrt_mufu(r2);
                if (self) inv = (sbase + s == tix[k]) ? 0.f : inv;
                const float qi = h.w * inv;
                ap[k] += qi;
                const float c = qi * (inv * inv);
                ax[k] = fmaf(c, ex, ax[k]);
                ay[k] = fmaf(c, ey, ay[k]);
                az[k] = fmaf(c, ez, az[k]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int k = 0; k < K; ++k) {
        fold(Hp[k], Lp[k], ap[k]);
        fold(Hx[k], Lx[k], ax[k]);
        fold(Hy[k], Ly[k], ay[k]);
        fold(Hz[k], Lz[k], az[k]);
      }
      __syncthreads();
    }
    float4* out = fpart + 2 * (S.part + (long long)it.z * n);
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (tix[k] < n) {
        out[2 * tix[k]] = make_float4(Hp[k], Hx[k], Hy[k], Hz[k]);
        out[2 * tix[k] + 1] = make_float4(Lp[k], Lx[k], Ly[k], Lz[k]);
      }
  }
}

// the pair configurations of k_pairs.cu (same items and target blocks)
#define HSMA_FIELD_CONFIGS(X) \
  X(0, 128, 4) X(1, 128, 2) X(2, 256, 2) X(3, 256, 4) X(4, 64, 4) X(5, 128, 1) X(6, 256, 1) X(7, 128, 8) \
  X(8, 64, 2) X(9, 64, 1) X(10, 32, 2) X(11, 32, 4)

int field_f32_occupancy(int cfg)
{
  int b = 0;
  switch (pair_kernel_of(cfg)) {
#define HSMA_FCFG_OCC(i, nt, k) \
  case i: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_field_f32<nt, k>, nt, 0); break;
    HSMA_FIELD_CONFIGS(HSMA_FCFG_OCC)
#undef HSMA_FCFG_OCC
    default: break;
  }
  return b;
}

int field_f64_occupancy();

void launch_field_f32(int cfg, int grid, const SysDev* sys, PairWork w1, PairWork w2, const float4* src_hi,
                      const float4* src_lo, const float4* surf_a, const float4* surf_b, const float4* boxes,
                      float4* fpart, cudaStream_t st, bool pdl)
{
  switch (pair_kernel_of(cfg)) {
#define HSMA_FCFG_LAUNCH(i, nt, k)                                                                        \
  case i:                                                                                                 \
    launch_k(k_field_f32<nt, k>, grid, nt, 0, st, pdl, sys, w1, w2, src_hi, src_lo, surf_a, surf_b, boxes, \
             fpart);                                                                                     \
    break;
    HSMA_FIELD_CONFIGS(HSMA_FCFG_LAUNCH)
#undef HSMA_FCFG_LAUNCH
    default: break;
  }
}

// ---------------------------------------------------------------------------------------
// FP64 comparator: one target per thread, plain staged loads.
constexpr int kF64FThreads = kF64TargetsPerBlock;

__global__ __launch_bounds__(kF64FThreads) void k_field_f64(const SysDev* __restrict__ sys, PairWork w1,
                                                            PairWork w2, const dbl4* __restrict__ src64,
                                                            const dbl4* __restrict__ surf64_a,
                                                            const double* __restrict__ surf64_b,
                                                            dbl4* __restrict__ fpart64)
{
  __shared__ dbl4 shA[kF64FThreads];
  __shared__ double shB[kF64FThreads];
  __shared__ int s_item, s_list;
  const int tid = threadIdx.x;
  int list = 0;
  bool first_fetch = true;
  grid_dependency_wait();  // (a programmatic launch: the records and counters of the pass)
  for (;;) {
    if (tid == 0) next_pair_item(w1, w2, list, first_fetch, s_item, s_list);
    first_fetch = false;
    __syncthreads();
    const int item = s_item;
    list = s_list;
    __syncthreads();
    if (list > 1) break;
    const int4 it = (list == 0 ? w1.items : w2.items)[item];
    const SysDev& S = sys[it.x];
    const int n = S.n;
    const int i = it.y * kF64FThreads + tid;
    const dbl4 tg = src64[S.src + (i < n ? i : it.y * kF64FThreads)];
    const FChunk ch = field_chunk(S, it.z);
    const double Rt = S.Rtau, rm = S.Rtau - 0.5 * S.dy, rp = S.Rtau + 0.5 * S.dy;
    double ap = 0.0, ax = 0.0, ay = 0.0, az = 0.0;
    for (int t0 = 0; t0 < ch.count; t0 += kF64FThreads) {
      const int cnt = min(kF64FThreads, ch.count - t0);
      if (tid < cnt) {
        if (ch.type == 2) {
          shA[tid] = surf64_a[ch.off + t0 + tid];
          shB[tid] = surf64_b[ch.off + t0 + tid];
        } else {
          shA[tid] = src64[ch.off + t0 + tid];
        }
      }
      __syncthreads();
      if (ch.type == 2) {
        for (int s = 0; s < cnt; ++s) {
          const dbl4 y = shA[s];
          const double D = shB[s];
          const double ux = tg.x - y.x, uy = tg.y - y.y, uz = tg.z - y.z;
          const double d = sqrt(ux * ux + uy * uy + uz * uz);
          const double c = y.w / (d * d * d);
          ap += y.w / d;
          ax += c * ux;
          ay += c * uy;
          az += c * uz;
          const double rho = sqrt(y.x * y.x + y.y * y.y + y.z * y.z);
          const double hx = y.x / rho, hy = y.y / rho, hz = y.z / rho;
          const double mx = tg.x - rm * hx, my = tg.y - rm * hy, mz = tg.z - rm * hz;
          const double px = tg.x - rp * hx, py = tg.y - rp * hy, pz = tg.z - rp * hz;
          const double dm = sqrt(mx * mx + my * my + mz * mz);
          const double dp = sqrt(px * px + py * py + pz * pz);
          const double xy = tg.x * hx + tg.y * hy + tg.z * hz;
          ap += D * 2.0 * (Rt - xy) / (dp * dm * (dp + dm));
          const double dm3 = dm * dm * dm, dp3 = dp * dp * dp;
          const double f = 2.0 * (Rt - xy) * (dp * dp + dp * dm + dm * dm) / ((dp + dm) * dm3 * dp3);
          ax += D * (hx / dm3 + px * f);
          ay += D * (hy / dm3 + py * f);
          az += D * (hz / dm3 + pz * f);
        }
      } else {
        const int sb = ch.first + t0;
        for (int s = 0; s < cnt; ++s) {
          const dbl4 h = shA[s];
          if (ch.type == 0 && sb + s == i) continue;
          // separately rounded IEEE operations, as in the potential (a charge next to its own
          // Kelvin image is an ill-conditioned distance)
          const double dx = tg.x - h.x, dy = tg.y - h.y, dz = tg.z - h.z;
          const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
          const double d = sqrt(r2);
          ap += h.w / d;
          const double c = h.w / (r2 * d);
          ax += c * dx;
          ay += c * dy;
          az += c * dz;
        }
      }
      __syncthreads();
    }
    if (i < n) fpart64[S.part + (long long)it.z * n + i] = make_dbl4(ap, ax, ay, az);
  }
}

int field_f64_occupancy()
{
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_field_f64, kF64FThreads, 0);
  return b;
}

void launch_field_f64(int grid, const SysDev* sys, PairWork w1, PairWork w2, const dbl4* src64,
                      const dbl4* surf64_a, const double* surf64_b, dbl4* fpart64, cudaStream_t st, bool pdl)
{
  launch_k(k_field_f64, grid, kF64FThreads, 0, st, pdl, sys, w1, w2, src64, surf64_a, surf64_b, fpart64);
}

// ---------------------------------------------------------------------------------------
// Coulomb (real chunks) and reaction (Kelvin + surface chunks + the centre constant, which has
// no field) potentials and fields; energies as in k_reduce (per-system completion).
constexpr int kFRedLanes = 8;
constexpr int kFRedTargets = 32;
constexpr int kFRedThreads = kFRedLanes * kFRedTargets;
static_assert(kFRedTargets == kReduceTargetsPerBlock, "the field reduction walks the reduce items");

__device__ __forceinline__ df dshfl(df v, int o)
{
  return df_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

// Adds the (hi, lo) partials of chunks k0, k0 + kFRedLanes, ... < k1 in ascending order, two
// chunks' loads in flight ahead of the additions.
__device__ __forceinline__ void sum_field_chunks(const float4* __restrict__ b, long long n, int k0, int k1, df* acc)
{
  int k = k0;
  for (; k + kFRedLanes < k1; k += 2 * kFRedLanes) {
    const float4 h0 = b[2 * (long long)k * n], l0 = b[2 * (long long)k * n + 1];
    const float4 h1 = b[2 * (long long)(k + kFRedLanes) * n], l1 = b[2 * (long long)(k + kFRedLanes) * n + 1];
    acc[0] = acc[0] + df_make(h0.x, l0.x);
    acc[1] = acc[1] + df_make(h0.y, l0.y);
    acc[2] = acc[2] + df_make(h0.z, l0.z);
    acc[3] = acc[3] + df_make(h0.w, l0.w);
    acc[0] = acc[0] + df_make(h1.x, l1.x);
    acc[1] = acc[1] + df_make(h1.y, l1.y);
    acc[2] = acc[2] + df_make(h1.z, l1.z);
    acc[3] = acc[3] + df_make(h1.w, l1.w);
  }
  for (; k < k1; k += kFRedLanes) {
    const float4 h = b[2 * (long long)k * n], l = b[2 * (long long)k * n + 1];
    acc[0] = acc[0] + df_make(h.x, l.x);
    acc[1] = acc[1] + df_make(h.y, l.y);
    acc[2] = acc[2] + df_make(h.z, l.z);
    acc[3] = acc[3] + df_make(h.w, l.w);
  }
}

__global__ __launch_bounds__(kFRedThreads) void k_reduce_field(
    const SysDev* __restrict__ sys, const int* __restrict__ sel, const int2* __restrict__ sel_rng, int nsel,
    const int2* __restrict__ items, const float4* __restrict__ fpart, const dbl4* __restrict__ fpart64, int prec,
    const double* __restrict__ q, const int* __restrict__ perm, const double* __restrict__ r0,
    double* __restrict__ phi_c, double* __restrict__ phi_r, double* __restrict__ phi_t, double* __restrict__ E_c,
    double* __restrict__ E_r, double* __restrict__ E_t, double* __restrict__ epart, double* __restrict__ energy,
    unsigned int* __restrict__ counter, int* __restrict__ status)
{
  __shared__ double red[2][kFRedThreads / 32];
  __shared__ bool last;
  __shared__ int s_r;
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int n = S.n;
  const int sub = threadIdx.x % kFRedLanes;
  const int i = it.y * kFRedTargets + threadIdx.x / kFRedLanes;
  const int nch = S.ncr + S.nck + S.ncs;
  double c[4] = {0.0, 0.0, 0.0, 0.0}, r[4] = {0.0, 0.0, 0.0, 0.0};
  if (prec == HSMA_FP64) {
    if (i < n) {
      const dbl4* b = fpart64 + S.part + i;
      for (int k = sub; k < nch; k += kFRedLanes) {
        const dbl4 v = b[(long long)k * n];
        double* a = k < S.ncr ? c : r;
        a[0] += v.x;
        a[1] += v.y;
        a[2] += v.z;
        a[3] += v.w;
      }
    }
    for (int o = 1; o < kFRedLanes; o <<= 1)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        c[m] += __shfl_xor_sync(0xffffffffu, c[m], o);
        r[m] += __shfl_xor_sync(0xffffffffu, r[m], o);
      }
  } else {
    df cc[4], rr[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) cc[m] = rr[m] = df_make(0.f, 0.f);
    if (i < n) {
      const float4* b = fpart + 2 * (S.part + i);
      sum_field_chunks(b, n, sub, S.ncr, cc);
      sum_field_chunks(b, n, S.ncr + sub, nch, rr);
    }
    for (int o = 1; o < kFRedLanes; o <<= 1)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        cc[m] = cc[m] + dshfl(cc[m], o);
        rr[m] = rr[m] + dshfl(rr[m], o);
      }
    if (sub == 0)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        c[m] = df_to_double(cc[m]);
        r[m] = df_to_double(rr[m]);
      }
  }
  double et = 0.0, er = 0.0;
  if (i < n && sub == 0) {
    r[0] += r0[it.x];
    const long long o = S.chg + perm[S.chg + i];
    phi_c[o] = c[0];
    phi_r[o] = r[0];
    phi_t[o] = c[0] + r[0];
#pragma unroll
    for (int m = 1; m < 4; ++m) {
      E_c[3 * o + m - 1] = c[m];
      E_r[3 * o + m - 1] = r[m];
      E_t[3 * o + m - 1] = c[m] + r[m];
    }
    bool bad = false;
#pragma unroll
    for (int m = 0; m < 4; ++m) bad = bad || !isfinite(c[m]) || !isfinite(r[m]);
    if (bad) atomicOr(status, kStNonFinite);
    const double qi = q[o];
    et = 0.5 * qi * (c[0] + r[0]);
    er = 0.5 * qi * r[0];
  }
  for (int o = 16; o > 0; o >>= 1) {
    et += __shfl_xor_sync(0xffffffffu, et, o);
    er += __shfl_xor_sync(0xffffffffu, er, o);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = et;
    red[1][warp] = er;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kFRedThreads / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    epart[2 * blockIdx.x] = a;
    epart[2 * blockIdx.x + 1] = b;
    __threadfence();
    int lo = 0, hi = nsel - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sel_rng[mid].x <= (int)blockIdx.x)
        lo = mid;
      else
        hi = mid - 1;
    }
    s_r = lo;
    const unsigned prev = atomicAdd(&counter[lo], 1u);
    last = (prev == (unsigned)sel_rng[lo].y - 1u);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const int rs = s_r;
  const int2 rg = sel_rng[rs];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < rg.y; k += kFRedThreads) {
    a += __ldcg(&epart[2 * (rg.x + k)]);
    b += __ldcg(&epart[2 * (rg.x + k) + 1]);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  __syncthreads();
  if (lane == 0) {
    red[0][warp] = a;
    red[1][warp] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double A = 0.0, B = 0.0;
    for (int w = 0; w < kFRedThreads / 32; ++w) {
      A += red[0][w];
      B += red[1][w];
    }
    energy[2 * sel[rs]] = A;
    energy[2 * sel[rs] + 1] = B;
    counter[rs] = 0u;
  }
}

void launch_reduce_field(const SysDev* sys, const int* sel, const int2* sel_rng, int nsel, const int2* items,
                         int nitems, const float4* fpart, const dbl4* fpart64, int prec, const double* q,
                         const int* perm, const double* r0, double* phi_c, double* phi_r, double* phi_t,
                         double* E_c, double* E_r, double* E_t, double* epart, double* energy, unsigned int* counter,
                         int* status, cudaStream_t st)
{
  if (nitems <= 0) return;
  k_reduce_field<<<nitems, kFRedThreads, 0, st>>>(sys, sel, sel_rng, nsel, items, fpart, fpart64, prec, q, perm, r0,
                                                  phi_c, phi_r, phi_t, E_c, E_r, E_t, epart, energy, counter, status);
}

}  // namespace hsma
