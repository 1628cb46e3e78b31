// FP32 pair-sum kernel (included by k_pairs.cu inside namespace hsma).
//
// Sources and targets are in the spatial order of k_order.cu.  A warp owns 32*K consecutive
// targets.
//
// Real and Kelvin sources (per warp, no CTA-wide synchronisation): the warp works in
// coordinates relative to an origin o at the centre of its targets' box; a target is held as
// the exact (hi, lo) FP32 split t' of x - o, a source as s' = fl(fl(x_hi - o) + x_lo) (within
// 2u |s'|, u = 2^-24).  The warp walks the chunk's 32-record source boxes; lane l loads record
// l of the next box while the current one is summed, and writes (-2 s', |s'|^2) and q of its
// record to the warp's shared buffer.  Per (warp, box) one of three forms is chosen, from
// X = (largest |t'|) + (largest |s'|) over the two boxes and their gap g (d >= g for every
// pair), so that each pair's relative error in 1/r stays below ~2.6e-6:
//   expanded  r^2 = |t'|^2 + |s'|^2 - 2 t'.s'   (1 FADD + 3 FFMA)   when X <= kExpRatio g:
//             the rounding of the expanded form, <= ~5 u X^2 in r^2, and the position errors,
//             <= 2 sqrt(3) u X / d, give <= 2.5 u (X/d)^2 + 3.5 u X/d relative in 1/r;
//   difference s = t'_hi - s',  r^2 = |s|^2      (3 + 3 operations)  when X <= kMidRatio g:
//             <= 2 sqrt(3) u X / d relative;
//   checked   the difference form where d >= X / kMidRatio; the rare closer pairs (r^2 below
//             that bound, the self pair included) are marked in a per-target mask in the loop
//             and added afterwards in the exact hi/lo form: t' and s' as exact splits from the
//             raw records, s = (t'_hi - s'_hi) + (t'_lo - s'_lo), accurate to FP32 rounding at
//             any distance (a charge next to its own Kelvin image); the self pair gets
//             r^2 = +inf, i.e. no contribution.
// Each pair then costs one MUFU rsqrt and one FFMA.
//
// Surface sources (CTA tiles staged with cp.async): monopole and dipole share one rsqrt; the
// dipole pair in its dy -> 0 limit.  Absolute FP32 coordinates: d >= tau a for every target.
//
// Each target keeps an FP32 partial per group of sources, folded into an (hi, lo) two-sum pair.

// ratios of the form choice (see above): 2.5 u 3.6^2 + 3.5 u 3.6 = 2.7e-6 and
// 2 sqrt(3) u 12 = 2.5e-6
constexpr float kExpRatio = 3.6f;
constexpr float kMidRatio = 12.0f;
constexpr int kFoldBoxes = 4;  // boxes summed in FP32 before a two-sum fold

enum : int { kFormExp = 0, kFormMid = 1, kFormChecked = 2 };

// exact x = hi + lo of (a + b) for FP32 a, b (Knuth's two-sum)
__device__ __forceinline__ void two_sum_f(float a, float b, float& s, float& e)
{
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (xh + xl) - o as an (hi, lo) pair: two-sum of xh - o, the low parts added, renormalised
__device__ __forceinline__ void rel_split(float xh, float xl, float o, float& h, float& l)
{
  float s, e;
  two_sum_f(xh, -o, s, e);
  const float t = e + xl;
  h = s + t;
  l = t - (h - s);
}

// The exact squared distance of a close pair (the checked form's fallback): target and source
// as exact splits relative to the origin, from their raw (hi, lo) records.
__device__ __forceinline__ float exact_r2(float4 th, float4 tl, float4 sh, float4 sl, float ox, float oy, float oz)
{
  float txh, txl, tyh, tyl, tzh, tzl, sxh, sxl, syh, syl, szh, szl;
  rel_split(th.x, tl.x, ox, txh, txl);
  rel_split(th.y, tl.y, oy, tyh, tyl);
  rel_split(th.z, tl.z, oz, tzh, tzl);
  rel_split(sh.x, sl.x, ox, sxh, sxl);
  rel_split(sh.y, sl.y, oy, syh, syl);
  rel_split(sh.z, sl.z, oz, szh, szl);
  const float ex = (txh - sxh) + (txl - sxl), ey = (tyh - syh) + (tyl - syl), ez = (tzh - szh) + (tzl - szl);
  float r2 = ex * ex;
  r2 = fmaf(ey, ey, r2);
  return fmaf(ez, ez, r2);
}

// One source of a box against the lane's K targets in one of the three forms.
template <int K, int FORM>
__device__ __forceinline__ void source_pairs(const float4 a, const float q, const float (&tx)[K], const float (&ty)[K],
                                             const float (&tz)[K], const float (&c)[K], float (&acc)[K])
{
#pragma unroll
  for (int k = 0; k < K; ++k) {
    float r2;
    if (FORM == kFormExp) {
      r2 = fmaf(tx[k], a.x, fmaf(ty[k], a.y, fmaf(tz[k], a.z, a.w + c[k])));
    } else {
      // 0.5 a.x = -s'_x exactly: one rounding, as t'_hi - s'
      const float dx = fmaf(0.5f, a.x, tx[k]), dy = fmaf(0.5f, a.y, ty[k]), dz = fmaf(0.5f, a.z, tz[k]);
      r2 = dx * dx;
      r2 = fmaf(dy, dy, r2);
      r2 = fmaf(dz, dz, r2);
    }
    acc[k] = fmaf(q, rsqrt_mufu(r2), acc[k]);
  }
}

// A box of cnt sources (the warp's buffer) in the expanded or the difference form.
template <int K, int FORM>
__device__ __forceinline__ void box_pairs(const float4* __restrict__ bA, const float* __restrict__ bQ, int cnt,
                                          const float (&tx)[K], const float (&ty)[K], const float (&tz)[K],
                                          const float (&c)[K], float (&acc)[K])
{
  if (cnt == kBox) {
#pragma unroll 8
    for (int s = 0; s < kBox; ++s) source_pairs<K, FORM>(bA[s], bQ[s], tx, ty, tz, c, acc);
  } else {
#pragma unroll 2
    for (int s = 0; s < cnt; ++s) source_pairs<K, FORM>(bA[s], bQ[s], tx, ty, tz, c, acc);
  }
}

// A box in the checked form: the difference form, where a pair with r^2 < thr2 adds nothing and
// is marked in its target's 32-bit source mask instead (no branch in the loop); the caller adds
// the marked pairs in the exact form.
template <int K, bool FULL>
__device__ __forceinline__ void box_pairs_checked(const float4* __restrict__ bA, const float* __restrict__ bQ, int cnt,
                                                  float thr2, const float (&tx)[K], const float (&ty)[K],
                                                  const float (&tz)[K], float (&acc)[K], unsigned (&mk)[K])
{
  const int ns = FULL ? kBox : cnt;
#pragma unroll(FULL ? 32 : 1)
  for (int s = 0; s < ns; ++s) {
    const float4 a = bA[s];
    const float q = bQ[s];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float dx = fmaf(0.5f, a.x, tx[k]), dy = fmaf(0.5f, a.y, ty[k]), dz = fmaf(0.5f, a.z, tz[k]);
      float r2 = dx * dx;
      r2 = fmaf(dy, dy, r2);
      r2 = fmaf(dz, dz, r2);
      const bool close = r2 < thr2;
      if (close) mk[k] |= 1u << s;
      const float inv = rsqrt_mufu(r2);
      acc[k] = fmaf(q, close ? 0.f : inv, acc[k]);
    }
  }
}

// registers per thread the kernel is compiled for (launch bounds: resident CTAs per SM), so
// that the warps of several CTAs share each SM sub-partition's MUFU
template <int NT, int K>
constexpr int pair_min_blocks()
{
  constexpr int regs = K >= 8 ? 168 : (K >= 4 ? 128 : 96);
  return 65536 / (NT * regs) > 0 ? 65536 / (NT * regs) : 1;
}

template <int NT, int K>
__global__ __launch_bounds__(NT, pair_min_blocks<NT, K>()) void k_pairs_f32(const SysDev* __restrict__ sys, PairWork w1, PairWork w2,
                                                  const float4* __restrict__ src_hi,
                                                  const float4* __restrict__ src_lo,
                                                  const float4* __restrict__ surf_a,
                                                  const float4* __restrict__ surf_b,
                                                  const float4* __restrict__ boxes, float2* __restrict__ part)
{
  static_assert(NT % 32 == 0, "whole warps");
  constexpr int NW = NT / 32;
  __shared__ __align__(16) float4 shA[2][NT];  // surface tiles
  __shared__ __align__(16) float4 shB[2][NT];
  __shared__ __align__(16) float4 wA[NW][32];  // per warp: (-2 s', |s'|^2) of the current box
  __shared__ float wQ[NW][32];                 // per warp: q of the current box
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
    const int w0 = t0 + warp * 32 * K;  // the warp's targets are [w0, w0 + 32 K)
    const ChunkInfo ch = decode_chunk(S, it.z);
    float H[K], L[K];
#pragma unroll
    for (int k = 0; k < K; ++k) H[k] = L[k] = 0.f;
    int tix[K];
#pragma unroll
    for (int k = 0; k < K; ++k) tix[k] = w0 + k * 32 + lane;

    if (ch.type == 2) {
      // ---- surface sources: CTA tiles -------------------------------------------------
      const float4* gA = surf_a + ch.off;
      const float4* gB = surf_b + ch.off;
      const int ntiles = (ch.count + NT - 1) / NT;
      if (tid < ch.count) {
        cp_async16(&shA[0][tid], gA + tid);
        cp_async16(&shB[0][tid], gB + tid);
      }
      cp_async_commit();
      float txh[K], tyh[K], tzh[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float4 h = src_hi[S.src + (tix[k] < n ? tix[k] : t0)];
        txh[k] = h.x; tyh[k] = h.y; tzh[k] = h.z;
      }
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
        float acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = 0.f;
#pragma unroll 2
        for (int s = 0; s < cnt; ++s) {
          const float4 y = A[s];
          const float Dp = B[s].x;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const float dx = txh[k] - y.x, dy = tyh[k] - y.y, dz = tzh[k] - y.z;
            float r2 = dx * dx;
            r2 = fmaf(dy, dy, r2);
            r2 = fmaf(dz, dz, r2);
            const float inv = rsqrt_mufu(r2);
            float dot = dx * y.x;
            dot = fmaf(dy, y.y, dot);
            dot = fmaf(dz, y.z, dot);
            const float u = dot * (inv * inv);
            const float v = fmaf(Dp, u, y.w);
            acc[k] = fmaf(v, inv, acc[k]);
          }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) {
          const float s = H[k] + acc[k];
          const float bp = s - H[k];
          L[k] += (H[k] - (s - bp)) + (acc[k] - bp);
          H[k] = s;
        }
        __syncthreads();
      }
    } else {
      // ---- real / Kelvin sources: per warp, relative coordinates ---------------------
      const float4* gh = src_hi + ch.off;
      const float4* gl = src_lo + ch.off;
      const int nb = (ch.count + kBox - 1) / kBox;
      // the first box's record is in flight while the targets load
      float4 rh = make_float4(0.f, 0.f, 0.f, 0.f), rl = rh;
      if (lane < ch.count) {
        rh = __ldg(gh + lane);
        rl = __ldg(gl + lane);
      }
      float tx[K], ty[K], tz[K], c[K];
      float wmnx = 3.0e38f, wmny = 3.0e38f, wmnz = 3.0e38f, wmxx = -3.0e38f, wmxy = -3.0e38f, wmxz = -3.0e38f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float4 h = src_hi[S.src + (tix[k] < n ? tix[k] : t0)];
        tx[k] = h.x; ty[k] = h.y; tz[k] = h.z;
        wmnx = fminf(wmnx, h.x); wmny = fminf(wmny, h.y); wmnz = fminf(wmnz, h.z);
        wmxx = fmaxf(wmxx, h.x); wmxy = fmaxf(wmxy, h.y); wmxz = fmaxf(wmxz, h.z);
      }
      // box of the warp's targets (hi coordinates) and its centre, the origin o
      for (int o = 16; o > 0; o >>= 1) {
        wmnx = fminf(wmnx, __shfl_xor_sync(0xffffffffu, wmnx, o));
        wmny = fminf(wmny, __shfl_xor_sync(0xffffffffu, wmny, o));
        wmnz = fminf(wmnz, __shfl_xor_sync(0xffffffffu, wmnz, o));
        wmxx = fmaxf(wmxx, __shfl_xor_sync(0xffffffffu, wmxx, o));
        wmxy = fmaxf(wmxy, __shfl_xor_sync(0xffffffffu, wmxy, o));
        wmxz = fmaxf(wmxz, __shfl_xor_sync(0xffffffffu, wmxz, o));
      }
      const float ox = 0.5f * (wmnx + wmxx), oy = 0.5f * (wmny + wmxy), oz = 0.5f * (wmnz + wmxz);
      // targets relative to o (the hi part of the exact split), |t'_hi|^2, largest |t'|
      float rw2 = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float4 l = src_lo[S.src + (tix[k] < n ? tix[k] : t0)];
        float lo;
        rel_split(tx[k], l.x, ox, tx[k], lo);
        rel_split(ty[k], l.y, oy, ty[k], lo);
        rel_split(tz[k], l.z, oz, tz[k], lo);
        c[k] = fmaf(tx[k], tx[k], fmaf(ty[k], ty[k], tz[k] * tz[k]));
        rw2 = fmaxf(rw2, c[k]);
      }
      for (int o = 16; o > 0; o >>= 1) rw2 = fmaxf(rw2, __shfl_xor_sync(0xffffffffu, rw2, o));
      const float Rw = sqrtf(rw2) * 1.0001f + 1e-30f;
      const long long box0 = S.bb + (ch.type == 1 ? (n + kBox - 1) / kBox : 0) + ch.first / kBox;
      float4* bA = wA[warp];
      float* bQ = wQ[warp];
      float acc[K];
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = 0.f;
      int code = kFormChecked;  // lane l: form of box (group + l) and, for a checked box,
      float thr = 0.f;          // the squared distance below which a pair takes the exact form
      for (int b = 0; b < nb; ++b) {
        if ((b & 31) == 0) {
          // the forms of the next 32 boxes, one per lane
          const int bl = b + lane;
          code = kFormChecked;
          thr = 3.0e38f;
          if (bl < nb) {
            const float4 bmn = __ldg(&boxes[2 * (box0 + bl)]), bmx = __ldg(&boxes[2 * (box0 + bl) + 1]);
            const int s0 = ch.first + bl * kBox;
            const bool self = ch.type == 0 && s0 < w0 + 32 * K && w0 < s0 + kBox;
            if (!self && bmn.x > bmx.x) {
              code = kFormExp;  // only zero-strength records (images of centre charges)
            } else {
              const float gx = fmaxf(0.f, fmaxf(wmnx - bmx.x, bmn.x - wmxx));
              const float gy = fmaxf(0.f, fmaxf(wmny - bmx.y, bmn.y - wmxy));
              const float gz = fmaxf(0.f, fmaxf(wmnz - bmx.z, bmn.z - wmxz));
              const float g = sqrtf(gx * gx + gy * gy + gz * gz);
              const float ex = fmaxf(fabsf(bmn.x - ox), fabsf(bmx.x - ox));
              const float ey = fmaxf(fabsf(bmn.y - oy), fabsf(bmx.y - oy));
              const float ez = fmaxf(fabsf(bmn.z - oz), fabsf(bmx.z - oz));
              const float X = (Rw + sqrtf(ex * ex + ey * ey + ez * ez)) * 1.0001f;
              code = self ? kFormChecked
                          : (X <= kExpRatio * g ? kFormExp : (X <= kMidRatio * g ? kFormMid : kFormChecked));
              const float xm = X * (1.f / kMidRatio);
              // (at least the smallest normal number, so that r^2 = 0, a self pair among targets
              // of zero extent included, always takes the exact form)
              thr = fmaxf(xm * xm, 1.17549435e-38f);
            }
          }
        }
        const int form = __shfl_sync(0xffffffffu, code, b & 31);
        const float thr2 = __shfl_sync(0xffffffffu, thr, b & 31);
        const int cnt = min(kBox, ch.count - b * kBox);
        // the next box's record is loaded while this one is summed
        float4 nh = rh, nl = rl;
        if (b + 1 < nb && lane < ch.count - (b + 1) * kBox) {
          nh = __ldg(gh + (b + 1) * kBox + lane);
          nl = __ldg(gl + (b + 1) * kBox + lane);
        }
        __syncwarp();  // the previous box's sums have read the buffer
        if (lane < cnt) {
          const float sx = (rh.x - ox) + rl.x, sy = (rh.y - oy) + rl.y, sz = (rh.z - oz) + rl.z;
          bA[lane] = make_float4(-2.f * sx, -2.f * sy, -2.f * sz, fmaf(sx, sx, fmaf(sy, sy, sz * sz)));
          bQ[lane] = rh.w;
        }
        __syncwarp();
        if (form == kFormExp) {
          box_pairs<K, kFormExp>(bA, bQ, cnt, tx, ty, tz, c, acc);
        } else if (form == kFormMid) {
          box_pairs<K, kFormMid>(bA, bQ, cnt, tx, ty, tz, c, acc);
        } else {
          unsigned mk[K];
#pragma unroll
          for (int k = 0; k < K; ++k) mk[k] = 0u;
          if (cnt == kBox)
            box_pairs_checked<K, true>(bA, bQ, cnt, thr2, tx, ty, tz, acc, mk);
          else
            box_pairs_checked<K, false>(bA, bQ, cnt, thr2, tx, ty, tz, acc, mk);
          // the marked close pairs in the exact hi/lo form from the raw records (the self pair:
          // no term)
          const int sb = ch.first + b * kBox;
#pragma unroll
          for (int k = 0; k < K; ++k) {
            unsigned m = mk[k];
            while (m) {
              const int sx = __ffs(m) - 1;
              m &= m - 1u;
              const int ti = tix[k] < n ? tix[k] : t0;
              float r2 = exact_r2(src_hi[S.src + ti], src_lo[S.src + ti], __ldg(gh + b * kBox + sx),
                                  __ldg(gl + b * kBox + sx), ox, oy, oz);
              if (ch.type == 0 && sb + sx == tix[k]) r2 = __int_as_float(0x7f800000);  // +inf
              const float q = bQ[sx];
              acc[k] = fmaf(q, rsqrt_mufu(r2), acc[k]);
            }
          }
        }
        if ((b + 1) % kFoldBoxes == 0 || b + 1 == nb) {
          // two-sum fold of the group's partial
#pragma unroll
          for (int k = 0; k < K; ++k) {
            const float s = H[k] + acc[k];
            const float bp = s - H[k];
            L[k] += (H[k] - (s - bp)) + (acc[k] - bp);
            H[k] = s;
            acc[k] = 0.f;
          }
        }
        rh = nh;
        rl = nl;
      }
    }
    float2* out = part + S.part + (long long)it.z * n;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (tix[k] < n) out[tix[k]] = make_float2(H[k], L[k]);
  }
}
