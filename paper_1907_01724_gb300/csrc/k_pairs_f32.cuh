// FP32 pair-sum kernel (included by k_pairs.cu inside namespace hsma).
//
// Work is split among warps, not CTAs: every warp pulls its own items and never waits for the
// other warps of its CTA.  Records and targets are in the spatial order of k_order.cu.
//
// Real and Kelvin items (system, block b, chunk c >= b): blocks and chunks are the same runs of
// S.chunk sorted charges.  The warp takes the block's targets in groups of 32 K (K per lane)
// and, for each group, walks the chunk's 32-record source boxes.
//  * Coordinates relative to an origin o at the centre of the group's box: a target is held as
//    the exact (hi, lo) FP32 split t' of x - o, a source as s' = fl(fl(x_hi - o) + x_lo) (within
//    2u |s'|, u = 2^-24).  Lane l loads record l of the next box while the current one is
//    summed, and writes (-2 s', |s'|^2) and q of its record to the warp's buffer.
//  * Per (group, box) one of three forms, from X = (largest |t'|) + (largest |s'|) over the two
//    boxes and their gap g (d >= g for every pair), so that each pair's relative error in 1/r
//    stays below ~2.7e-6:
//      expanded    r^2 = |t'|^2 + |s'|^2 - 2 t'.s'  (1 FADD + 3 FFMA)  when X <= kExpRatio g:
//                  the rounding of the expanded form, <= ~5 u X^2 in r^2, and the position
//                  errors, <= 2 sqrt(3) u X / d, give <= 2.5 u (X/d)^2 + 3.5 u X/d;
//      difference  s = t'_hi - s', r^2 = |s|^2      (3 + 3 operations) when X <= kMidRatio g:
//                  <= 2 sqrt(3) u X / d;
//      checked     the difference form where d >= X / kMidRatio; the rare closer pairs (r^2
//                  below that bound, the self pair included) are marked in a mask in the loop
//                  and added afterwards in the exact hi/lo form: t' and s' as exact splits from
//                  the raw records, s = (t'_hi - s'_hi) + (t'_lo - s'_lo), accurate to FP32
//                  rounding at any distance (a charge next to its own Kelvin image); the self
//                  pair gets r^2 = +inf, i.e. no contribution.  The box's sources are split
//                  once, by the lanes that hold their records, into the warp's shared memory,
//                  and each lane splits its targets once per box, so a marked pair costs no
//                  global load (near the interface most boxes of a block and its own images'
//                  chunk have marked pairs).
//  * Off-diagonal items (c > b) are evaluated once per unordered pair, both ways.  Real pairs by
//    Newton's third law: 1/|x_i - x_j| serves i's term from j and j's term from i.  Kelvin pairs
//    by Kelvin inversion, |x_j - x_i*| = |x_i - x_j*| |x_j| / |x_i| (x* = a^2 x / |x|^2): the
//    target i's term from j's image is q_K,j / |x_i - x_j*|, and j's term from i's image is
//    (q_K,i |x_i|) (1 / |x_i - x_j*|) (1 / |x_j|); k_images stores q_K,i |x_i| with the real
//    record and 1 / |x_j| with the Kelvin record.  In a box the lanes walk a ring: at step j
//    lane l takes source (l + j) mod 32 and hands that source's running sum of the transposed
//    terms to lane l - 1, so after 32 steps lane l holds its source's sum over the group's
//    targets; the sums are kept per source as (hi, lo) pairs in the warp's shared memory and
//    written, for the block's slot, at the end of the item.  The diagonal item (c = b) is
//    evaluated one way and skips the self pair.
//
// Surface items (system, group of 32 K targets, surface chunk): points staged per warp the same
// way; monopole and dipole share one rsqrt, the dipole pair in its dy -> 0 limit; absolute FP32
// coordinates (d >= tau a for every target).
//
// Each target keeps an FP32 partial per group of boxes, folded into an (hi, lo) two-sum pair.

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

// (H, L) += v (two-sum)
__device__ __forceinline__ void fold_two_sum(float& H, float& L, float v)
{
  const float s = H + v;
  const float bp = s - H;
  L += (H - (s - bp)) + (v - bp);
  H = s;
}

// The exact form of a close pair (the checked form's fallback): coordinates as exact (hi, lo)
// splits relative to the origin, from their raw (hi, lo) records; e = (xh, xl, yh, yl, zh, zl).
__device__ __forceinline__ void exact_split(float4 h, float4 l, float ox, float oy, float oz, float (&e)[6])
{
  rel_split(h.x, l.x, ox, e[0], e[1]);
  rel_split(h.y, l.y, oy, e[2], e[3]);
  rel_split(h.z, l.z, oz, e[4], e[5]);
}

// squared distance of a target and a source from their exact splits: the differences of the hi
// and of the lo parts, summed per coordinate, accurate to FP32 rounding at any distance
__device__ __forceinline__ float exact_r2(const float (&t)[6], float sxh, float sxl, float syh, float syl,
                                          float szh, float szl)
{
  const float ex = (t[0] - sxh) + (t[1] - sxl), ey = (t[2] - syh) + (t[3] - syl), ez = (t[4] - szh) + (t[5] - szl);
  float r2 = ex * ex;
  r2 = fmaf(ey, ey, r2);
  return fmaf(ez, ez, r2);
}

// Lane l writes the exact split of its record (rh, rl) of the current box to column l of E (for
// l < cnt; the other columns are never read: past the box no pair is marked), then the warp syncs.
__device__ __forceinline__ void stage_exact_sources(float (*E)[kBox], int lane, int cnt, float4 rh, float4 rl,
                                                    float ox, float oy, float oz)
{
  if (lane < cnt) {
    float e[6];
    exact_split(rh, rl, ox, oy, oz, e);
#pragma unroll
    for (int c = 0; c < 6; ++c) E[c][lane] = e[c];
  }
  __syncwarp();
}

// Squared distance of a target (relative hi part tx, ty, tz and |t'|^2 = c) to a buffered
// source a = (-2 s', |s'|^2) in the expanded or the difference form.
template <int FORM>
__device__ __forceinline__ float pair_r2(const float4 a, float tx, float ty, float tz, float c)
{
  if (FORM == kFormExp) return fmaf(tx, a.x, fmaf(ty, a.y, fmaf(tz, a.z, a.w + c)));
  // 0.5 a.x = -s'_x exactly: one rounding, as t'_hi - s'
  const float dx = fmaf(0.5f, a.x, tx), dy = fmaf(0.5f, a.y, ty), dz = fmaf(0.5f, a.z, tz);
  float r2 = dx * dx;
  r2 = fmaf(dy, dy, r2);
  return fmaf(dz, dz, r2);
}

// Packed FP32 over the target slots 2h and 2h + 1 of a lane (K even): one FFMA2 / FADD2 / FMUL2
// instruction (sm_100 and later) does an operation for both slots, rounded per component
// exactly as the scalar operation, so every sum is bitwise that of the scalar form.  The pair
// sums are issue-bound (the rsqrt, one MUFU operation per pair, stays scalar): packing halves
// the issue slots of their FP32 part.
__device__ __forceinline__ float2 bc2(float a) { return make_float2(a, a); }

template <int FORM>
__device__ __forceinline__ float2 pair_r2_x2(const float4 a, float2 tx, float2 ty, float2 tz, float2 c)
{
  if (FORM == kFormExp)
    return __ffma2_rn(tx, bc2(a.x), __ffma2_rn(ty, bc2(a.y), __ffma2_rn(tz, bc2(a.z), __fadd2_rn(bc2(a.w), c))));
  const float2 h = bc2(0.5f);
  const float2 dx = __ffma2_rn(h, bc2(a.x), tx), dy = __ffma2_rn(h, bc2(a.y), ty), dz = __ffma2_rn(h, bc2(a.z), tz);
  float2 r2 = __fmul2_rn(dx, dx);
  r2 = __ffma2_rn(dy, dy, r2);
  return __ffma2_rn(dz, dz, r2);
}

template <int K>
__device__ __forceinline__ void pack2(const float (&v)[K], float2 (&p)[K / 2])
{
#pragma unroll
  for (int h = 0; h < K / 2; ++h) p[h] = make_float2(v[2 * h], v[2 * h + 1]);
}
template <int K>
__device__ __forceinline__ void unpack2(const float2 (&p)[K / 2], float (&v)[K])
{
#pragma unroll
  for (int h = 0; h < K / 2; ++h) {
    v[2 * h] = p[h].x;
    v[2 * h + 1] = p[h].y;
  }
}

// One source of a box against the lane's K targets, packed (K even).
template <int K, int FORM>
__device__ __forceinline__ void pair_oneway_x2(const float4 a, float q, const float2 (&X)[K / 2],
                                               const float2 (&Y)[K / 2], const float2 (&Z)[K / 2],
                                               const float2 (&C)[K / 2], float2 (&A)[K / 2])
{
#pragma unroll
  for (int h = 0; h < K / 2; ++h) {
    const float2 r2 = pair_r2_x2<FORM>(a, X[h], Y[h], Z[h], C[h]);
    A[h] = __ffma2_rn(bc2(q), make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y)), A[h]);
  }
}

// One-way sums of a box (cnt sources of the warp's buffer) into the lane's K targets.
template <int K, int FORM>
__device__ __forceinline__ void box_oneway(const float4* __restrict__ bA, const float* __restrict__ bQ, int cnt,
                                           const float (&tx)[K], const float (&ty)[K], const float (&tz)[K],
                                           const float (&c)[K], float (&acc)[K])
{
  if constexpr (K % 2 == 0) {
    float2 X[K / 2], Y[K / 2], Z[K / 2], C[K / 2], A[K / 2];
    pack2<K>(tx, X);
    pack2<K>(ty, Y);
    pack2<K>(tz, Z);
    pack2<K>(c, C);
    pack2<K>(acc, A);
    if (cnt == kBox) {
#pragma unroll 4
      for (int s = 0; s < kBox; ++s) pair_oneway_x2<K, FORM>(bA[s], bQ[s], X, Y, Z, C, A);
    } else {
#pragma unroll 2
      for (int s = 0; s < cnt; ++s) pair_oneway_x2<K, FORM>(bA[s], bQ[s], X, Y, Z, C, A);
    }
    unpack2<K>(A, acc);
    return;
  }
  if (cnt == kBox) {
#pragma unroll 4
    for (int s = 0; s < kBox; ++s) {
      const float4 a = bA[s];
      const float q = bQ[s];
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = fmaf(q, rsqrt_mufu(pair_r2<FORM>(a, tx[k], ty[k], tz[k], c[k])), acc[k]);
    }
  } else {
#pragma unroll 2
    for (int s = 0; s < cnt; ++s) {
      const float4 a = bA[s];
      const float q = bQ[s];
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = fmaf(q, rsqrt_mufu(pair_r2<FORM>(a, tx[k], ty[k], tz[k], c[k])), acc[k]);
    }
  }
}

// One-way checked sums: a pair with r^2 < thr2 adds nothing and is marked in its target's mask
// (bit = source index).
template <int K>
__device__ __forceinline__ void box_oneway_checked(const float4* __restrict__ bA, const float* __restrict__ bQ,
                                                   int cnt, float thr2, const float (&tx)[K], const float (&ty)[K],
                                                   const float (&tz)[K], float (&acc)[K], unsigned (&mk)[K])
{
  if constexpr (K % 2 == 0) {
    float2 X[K / 2], Y[K / 2], Z[K / 2], A[K / 2];
    pack2<K>(tx, X);
    pack2<K>(ty, Y);
    pack2<K>(tz, Z);
    pack2<K>(acc, A);
#pragma unroll 4
    for (int s = 0; s < cnt; ++s) {
      const float4 a = bA[s];
      const float q = bQ[s];
#pragma unroll
      for (int h = 0; h < K / 2; ++h) {
        const float2 r2 = pair_r2_x2<kFormMid>(a, X[h], Y[h], Z[h], bc2(0.f));
        const bool c0 = r2.x < thr2, c1 = r2.y < thr2;
        if (c0) mk[2 * h] |= 1u << s;
        if (c1) mk[2 * h + 1] |= 1u << s;
        const float i0 = rsqrt_mufu(r2.x), i1 = rsqrt_mufu(r2.y);
        A[h] = __ffma2_rn(bc2(q), make_float2(c0 ? 0.f : i0, c1 ? 0.f : i1), A[h]);
      }
    }
    unpack2<K>(A, acc);
    return;
  }
#pragma unroll 4
  for (int s = 0; s < cnt; ++s) {
    const float4 a = bA[s];
    const float q = bQ[s];
#pragma unroll
    for (int k = 0; k < K; ++k) {
      const float r2 = pair_r2<kFormMid>(a, tx[k], ty[k], tz[k], 0.f);
      const bool close = r2 < thr2;
      if (close) mk[k] |= 1u << s;
      const float inv = rsqrt_mufu(r2);
      acc[k] = fmaf(q, close ? 0.f : inv, acc[k]);
    }
  }
}

// Both-way sums of a full or ragged box (the buffer holds the box twice, so that step j of lane
// l reads entry l + j, i.e. source (l + j) mod 32; entries past the box's sources are far-away
// zero charges).  The transposed terms go into kRing running sums, sum r taking the steps j = r
// (mod kRing): after step j it moves kRing lanes down, to the lane that takes the same source at
// step j + kRing.  After the 32 steps sum r of lane l belongs to source l + r; it is moved to
// lane l - r, and the lane's returned total belongs to source l.  (One sum: measured on GB300
// with 2, 4 and 8 interleaved sums, which shorten each sum's chain of dependent shuffles, the
// kernel was not faster.)  CHECKED: pairs with r^2 < thr2 add nothing either way and are marked
// in the target's mask (bit = step).
constexpr int kRing = 1;

template <int K, int FORM, bool CHECKED>
__device__ __forceinline__ float box_ring(const float4* __restrict__ bA, const float* __restrict__ bQ, int lane,
                                          float thr2, const float (&tx)[K], const float (&ty)[K],
                                          const float (&tz)[K], const float (&c)[K], const float (&wt)[K],
                                          float (&acc)[K], unsigned (&mk)[K])
{
  const float4* A = bA + lane;
  const float* Q = bQ + lane;
  float sacc[kRing];
#pragma unroll
  for (int r = 0; r < kRing; ++r) sacc[r] = 0.f;
  if constexpr (K % 2 == 0 && kRing == 1) {
    // packed: the targets' terms two slots per instruction; the transposed sum in slot order
    float2 X[K / 2], Y[K / 2], Z[K / 2], C[K / 2], AC[K / 2];
    pack2<K>(tx, X);
    pack2<K>(ty, Y);
    pack2<K>(tz, Z);
    pack2<K>(c, C);
    pack2<K>(acc, AC);
    float sa = 0.f;
#pragma unroll 8
    for (int j = 0; j < kBox; ++j) {
      const float4 a = A[j];
      const float q = Q[j];
#pragma unroll
      for (int h = 0; h < K / 2; ++h) {
        const float2 r2 = pair_r2_x2<FORM>(a, X[h], Y[h], Z[h], C[h]);
        float i0 = rsqrt_mufu(r2.x), i1 = rsqrt_mufu(r2.y);
        if (CHECKED) {
          const bool c0 = r2.x < thr2, c1 = r2.y < thr2;
          if (c0) mk[2 * h] |= 1u << j;
          if (c1) mk[2 * h + 1] |= 1u << j;
          i0 = c0 ? 0.f : i0;
          i1 = c1 ? 0.f : i1;
        }
        AC[h] = __ffma2_rn(bc2(q), make_float2(i0, i1), AC[h]);
        sa = fmaf(wt[2 * h], i0, sa);
        sa = fmaf(wt[2 * h + 1], i1, sa);
      }
      sa = __shfl_sync(0xffffffffu, sa, (lane + 1) & 31);
    }
    unpack2<K>(AC, acc);
    return sa;
  }
#pragma unroll 8
  for (int j0 = 0; j0 < kBox; j0 += kRing) {
#pragma unroll
    for (int r = 0; r < kRing; ++r) {
      const int j = j0 + r;
      const float4 a = A[j];
      const float q = Q[j];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float r2 = pair_r2<FORM>(a, tx[k], ty[k], tz[k], c[k]);
        float inv = rsqrt_mufu(r2);
        if (CHECKED) {
          const bool close = r2 < thr2;
          if (close) mk[k] |= 1u << j;
          inv = close ? 0.f : inv;
        }
        acc[k] = fmaf(q, inv, acc[k]);
        sacc[r] = fmaf(wt[k], inv, sacc[r]);
      }
      sacc[r] = __shfl_sync(0xffffffffu, sacc[r], (lane + kRing) & 31);
    }
  }
  float tot = sacc[0];
#pragma unroll
  for (int r = 1; r < kRing; ++r) tot += __shfl_sync(0xffffffffu, sacc[r], (lane - r) & 31);
  return tot;
}

// registers per thread the kernel is compiled for (launch bounds: resident CTAs per SM), so
// that the warps of several CTAs share each SM sub-partition's MUFU
template <int NT, int K>
constexpr int pair_min_blocks()
{
  constexpr int regs = K >= 8 ? 168 : 128;
  return 65536 / (NT * regs) > 0 ? 65536 / (NT * regs) : 1;
}

// dynamic shared memory of a k_pairs_f32<NT, K> launch: per warp, kSymChunkMax (hi, lo) sums
// of the transposed terms
constexpr size_t pair_dyn_smem(int nt) { return (size_t)(nt / 32) * kSymChunkMax * sizeof(float2); }

template <int NT, int K>
__global__ __launch_bounds__(NT, pair_min_blocks<NT, K>()) void k_pairs_f32(const SysDev* __restrict__ sys,
                                                                          PairWork w1, PairWork w2,
                                                                          const float4* __restrict__ src_hi,
                                                                          const float4* __restrict__ src_lo,
                                                                          const float4* __restrict__ surf_a,
                                                                          const float4* __restrict__ surf_b,
                                                                          const float4* __restrict__ boxes,
                                                                          float2* __restrict__ part)
{
  static_assert(NT % 32 == 0, "whole warps");
  static_assert(kSymChunkMax % (32 * K) == 0, "blocks of whole target groups");
  constexpr int NW = NT / 32;
  constexpr int G = 32 * K;  // targets per group
  __shared__ __align__(16) float4 wA[NW][2 * kBox];  // relative source records of the box, twice
  __shared__ float wQ[NW][2 * kBox];                 // their charges
  __shared__ float wE[NW][6][kBox];                  // exact splits of a checked box's sources
  extern __shared__ float2 wP_all[];                 // per warp: (hi, lo) sums of transposed terms
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int worker = blockIdx.x * NW + warp;
  float4* bA = wA[warp];
  float* bQ = wQ[warp];
  float(*bE)[kBox] = wE[warp];
  float2* P = wP_all + (size_t)warp * kSymChunkMax;
  int list = 0;
  bool first_fetch = true;
  grid_dependency_wait();  // (a programmatic launch: the records and counters of the pass)

  for (;;) {
    // the warp's next item (lane 0 fetches, the warp follows)
    int item = 0;
    if (lane == 0) {
      int v = 0;
      if (list == 0) {
        v = first_fetch && worker < w1.first ? worker : pull_pair_item(w1);
        if (v < 0) list = 1;
      }
      if (list == 1) {
        v = pull_pair_item(w2);
        if (v < 0) list = 2;
      }
      item = v;
    }
    item = __shfl_sync(0xffffffffu, item, 0);
    list = __shfl_sync(0xffffffffu, list, 0);
    first_fetch = false;
    if (list > 1) break;
    const int4 it = (list == 0 ? w1.items : w2.items)[item];
    const SysDev& S = sys[it.x];
    const int n = S.n;
    const ChunkInfo ch = decode_chunk(S, it.z);

    if (ch.type == 2) {
      // ---- surface item: one group of targets against a chunk of surface points ----------
      const int g0 = it.y * G;
      float tx[K], ty[K], tz[K], H[K], L[K], acc[K];
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = g0 + k * 32 + lane;
        const float4 h = src_hi[S.src + (i < n ? i : g0)];
        tx[k] = h.x; ty[k] = h.y; tz[k] = h.z;
        H[k] = L[k] = acc[k] = 0.f;
      }
      const float4* ga = surf_a + ch.off;
      const float4* gb = surf_b + ch.off;
      const int nb = (ch.count + kBox - 1) / kBox;
      float4 ra = make_float4(0.f, 0.f, 0.f, 0.f);
      float rd = 0.f;
      if (lane < ch.count) {
        ra = __ldg(ga + lane);
        rd = __ldg(gb + lane).x;
      }
      for (int b = 0; b < nb; ++b) {
        const int cnt = min(kBox, ch.count - b * kBox);
        float4 na = ra;
        float nd = rd;
        if (b + 1 < nb && lane < ch.count - (b + 1) * kBox) {
          na = __ldg(ga + (b + 1) * kBox + lane);
          nd = __ldg(gb + (b + 1) * kBox + lane).x;
        }
        __syncwarp();  // the previous box's sums have read the buffer
        if (lane < cnt) {
          bA[lane] = ra;
          bQ[lane] = rd;
        }
        __syncwarp();
        if constexpr (K % 2 == 0) {
          // packed (slots 2h, 2h + 1); t - y as t + (-y), the same rounding
          float2 X[K / 2], Y[K / 2], Z[K / 2], A[K / 2];
          pack2<K>(tx, X);
          pack2<K>(ty, Y);
          pack2<K>(tz, Z);
          pack2<K>(acc, A);
#pragma unroll 2
          for (int s = 0; s < cnt; ++s) {
            const float4 y = bA[s];
            const float Dp = bQ[s];
            const float2 yx = bc2(y.x), yy = bc2(y.y), yz = bc2(y.z);
#pragma unroll
            for (int h = 0; h < K / 2; ++h) {
              const float2 dx = __fadd2_rn(X[h], bc2(-y.x)), dy = __fadd2_rn(Y[h], bc2(-y.y)),
                           dz = __fadd2_rn(Z[h], bc2(-y.z));
              float2 r2 = __fmul2_rn(dx, dx);
              r2 = __ffma2_rn(dy, dy, r2);
              r2 = __ffma2_rn(dz, dz, r2);
              const float2 inv = make_float2(rsqrt_mufu(r2.x), rsqrt_mufu(r2.y));
              float2 dot = __fmul2_rn(dx, yx);
              dot = __ffma2_rn(dy, yy, dot);
              dot = __ffma2_rn(dz, yz, dot);
              const float2 u = __fmul2_rn(dot, __fmul2_rn(inv, inv));
              const float2 v = __ffma2_rn(bc2(Dp), u, bc2(y.w));
              A[h] = __ffma2_rn(v, inv, A[h]);
            }
          }
          unpack2<K>(A, acc);
        } else {
#pragma unroll 2
          for (int s = 0; s < cnt; ++s) {
            const float4 y = bA[s];
            const float Dp = bQ[s];
#pragma unroll
            for (int k = 0; k < K; ++k) {
              const float dx = tx[k] - y.x, dy = ty[k] - y.y, dz = tz[k] - y.z;
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
        }
        if ((b + 1) % kFoldBoxes == 0 || b + 1 == nb) {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            fold_two_sum(H[k], L[k], acc[k]);
            acc[k] = 0.f;
          }
        }
        ra = na;
        rd = nd;
      }
      float2* out = part + S.part + (long long)it.z * n;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = g0 + k * 32 + lane;
        if (i < n) out[i] = make_float2(H[k], L[k]);
      }
      continue;
    }

    // ---- real / Kelvin item: block blk of targets against chunk cb of sources ----------------
    const int blk = it.y;
    const int cb = ch.type == 0 ? it.z : it.z - S.ncr;
    const bool sym = cb > blk;
    const int tb0 = blk * S.chunk, tb1 = min(n, tb0 + S.chunk);
    const float4* gh = src_hi + ch.off;
    const float4* gl = src_lo + ch.off;
    const int nb = (ch.count + kBox - 1) / kBox;
    const long long box0 = S.bb + (ch.type == 1 ? (n + kBox - 1) / kBox : 0) + ch.first / kBox;
    if (sym) {
      for (int j = lane; j < ch.count; j += 32) P[j] = make_float2(0.f, 0.f);
    }
    for (int g0 = tb0; g0 < tb1; g0 += G) {
      // targets of the group (slots past the block repeat its first target, with no weight)
      float tx[K], ty[K], tz[K], c[K], wt[K], H[K], L[K], acc[K];
      float wmnx = 3.0e38f, wmny = 3.0e38f, wmnz = 3.0e38f, wmxx = -3.0e38f, wmxy = -3.0e38f, wmxz = -3.0e38f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = g0 + k * 32 + lane;
        const float4 h = src_hi[S.src + (i < tb1 ? i : g0)];
        tx[k] = h.x; ty[k] = h.y; tz[k] = h.z;
        wt[k] = h.w;
        H[k] = L[k] = acc[k] = 0.f;
        wmnx = fminf(wmnx, h.x); wmny = fminf(wmny, h.y); wmnz = fminf(wmnz, h.z);
        wmxx = fmaxf(wmxx, h.x); wmxy = fmaxf(wmxy, h.y); wmxz = fmaxf(wmxz, h.z);
      }
      for (int o = 16; o > 0; o >>= 1) {
        wmnx = fminf(wmnx, __shfl_xor_sync(0xffffffffu, wmnx, o));
        wmny = fminf(wmny, __shfl_xor_sync(0xffffffffu, wmny, o));
        wmnz = fminf(wmnz, __shfl_xor_sync(0xffffffffu, wmnz, o));
        wmxx = fmaxf(wmxx, __shfl_xor_sync(0xffffffffu, wmxx, o));
        wmxy = fmaxf(wmxy, __shfl_xor_sync(0xffffffffu, wmxy, o));
        wmxz = fmaxf(wmxz, __shfl_xor_sync(0xffffffffu, wmxz, o));
      }
      const float ox = 0.5f * (wmnx + wmxx), oy = 0.5f * (wmny + wmxy), oz = 0.5f * (wmnz + wmxz);
      float rw2 = 0.f;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = g0 + k * 32 + lane;
        const float4 l = src_lo[S.src + (i < tb1 ? i : g0)];
        // weight of the target as a source of the transposed terms: its charge (real pairs) or
        // q_K |x| (Kelvin pairs); none for a slot past the block
        wt[k] = i < tb1 ? (ch.type == 0 ? wt[k] : l.w) : 0.f;
        float lo;
        rel_split(tx[k], l.x, ox, tx[k], lo);
        rel_split(ty[k], l.y, oy, ty[k], lo);
        rel_split(tz[k], l.z, oz, tz[k], lo);
        c[k] = fmaf(tx[k], tx[k], fmaf(ty[k], ty[k], tz[k] * tz[k]));
        rw2 = fmaxf(rw2, c[k]);
      }
      for (int o = 16; o > 0; o >>= 1) rw2 = fmaxf(rw2, __shfl_xor_sync(0xffffffffu, rw2, o));
      const float Rw = sqrtf(rw2) * 1.0001f + 1e-30f;
      // the first box's record
      float4 rh = make_float4(0.f, 0.f, 0.f, 0.f), rl = rh;
      if (lane < ch.count) {
        rh = __ldg(gh + lane);
        rl = __ldg(gl + lane);
      }
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
            const bool self = ch.type == 0 && !sym && s0 < g0 + G && g0 < s0 + kBox;
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
        {
          float4 a = make_float4(-2.0e18f, 0.f, 0.f, 1.0e36f);  // past the box: far away, no charge
          float q = 0.f;
          if (lane < cnt) {
            const float sx = (rh.x - ox) + rl.x, sy = (rh.y - oy) + rl.y, sz = (rh.z - oz) + rl.z;
            a = make_float4(-2.f * sx, -2.f * sy, -2.f * sz, fmaf(sx, sx, fmaf(sy, sy, sz * sz)));
            q = rh.w;
          }
          bA[lane] = a;
          bA[lane + kBox] = a;
          bQ[lane] = q;
          bQ[lane + kBox] = q;
        }
        __syncwarp();
        unsigned mk[K];
#pragma unroll
        for (int k = 0; k < K; ++k) mk[k] = 0u;
        if (!sym) {
          if (form == kFormExp) {
            box_oneway<K, kFormExp>(bA, bQ, cnt, tx, ty, tz, c, acc);
          } else if (form == kFormMid) {
            box_oneway<K, kFormMid>(bA, bQ, cnt, tx, ty, tz, c, acc);
          } else {
            box_oneway_checked<K>(bA, bQ, cnt, thr2, tx, ty, tz, acc, mk);
            // the marked close pairs in the exact form (the self pair: no term); each lane
            // splits its own record of the box and its targets once
            unsigned any = 0u;
#pragma unroll
            for (int k = 0; k < K; ++k) any |= mk[k];
            if (__any_sync(0xffffffffu, any != 0u)) {
              stage_exact_sources(bE, lane, cnt, rh, rl, ox, oy, oz);
              const int sb = ch.first + b * kBox;
#pragma unroll
              for (int k = 0; k < K; ++k) {
                unsigned m = mk[k];
                if (!__any_sync(0xffffffffu, m != 0u)) continue;
                const int ti = g0 + k * 32 + lane;
                const int tr = ti < tb1 ? ti : g0;
                float te[6];
                exact_split(src_hi[S.src + tr], src_lo[S.src + tr], ox, oy, oz, te);
                while (m) {
                  const int sx = __ffs(m) - 1;
                  m &= m - 1u;
                  float r2 = exact_r2(te, bE[0][sx], bE[1][sx], bE[2][sx], bE[3][sx], bE[4][sx], bE[5][sx]);
                  if (ch.type == 0 && sb + sx == ti) r2 = __int_as_float(0x7f800000);  // +inf
                  acc[k] = fmaf(bQ[sx], rsqrt_mufu(r2), acc[k]);
                }
              }
            }
          }
        } else {
          float sacc;
          if (form == kFormExp) {
            sacc = box_ring<K, kFormExp, false>(bA, bQ, lane, thr2, tx, ty, tz, c, wt, acc, mk);
          } else if (form == kFormMid) {
            sacc = box_ring<K, kFormMid, false>(bA, bQ, lane, thr2, tx, ty, tz, c, wt, acc, mk);
          } else {
            sacc = box_ring<K, kFormMid, true>(bA, bQ, lane, thr2, tx, ty, tz, c, wt, acc, mk);
            unsigned any = 0u;
#pragma unroll
            for (int k = 0; k < K; ++k) any |= mk[k];
            if (__any_sync(0xffffffffu, any != 0u)) {
              // the marked close pairs, both ways, in the exact form.  Per target slot k a second
              // ring carries the transposed terms to their sources: it visits only the steps
              // where some lane has a marked pair, rotating the running sums by the steps between
              // them (lane l's sum belongs to source l + jc), and ends aligned (lane l: source l).
              stage_exact_sources(bE, lane, cnt, rh, rl, ox, oy, oz);
#pragma unroll
              for (int k = 0; k < K; ++k) {
                unsigned u = __reduce_or_sync(0xffffffffu, mk[k]);
                if (u == 0u) continue;
                const int ti = g0 + k * 32 + lane;
                const int tr = ti < tb1 ? ti : g0;
                float te[6];
                exact_split(src_hi[S.src + tr], src_lo[S.src + tr], ox, oy, oz, te);
                float fx = 0.f;
                int jc = 0;
                while (u) {
                  const int j = __ffs(u) - 1;
                  u &= u - 1u;
                  fx = __shfl_sync(0xffffffffu, fx, (lane + j - jc) & 31);
                  jc = j;
                  if ((mk[k] >> j) & 1u) {
                    const int sx = (lane + j) & 31;
                    const float inv =
                        rsqrt_mufu(exact_r2(te, bE[0][sx], bE[1][sx], bE[2][sx], bE[3][sx], bE[4][sx], bE[5][sx]));
                    acc[k] = fmaf(bQ[sx], inv, acc[k]);
                    fx = fmaf(wt[k], inv, fx);
                  }
                }
                sacc += __shfl_sync(0xffffffffu, fx, (lane + 32 - jc) & 31);
              }
            }
          }
          if (lane < cnt) {
            float2 p = P[b * kBox + lane];
            fold_two_sum(p.x, p.y, sacc);
            P[b * kBox + lane] = p;
          }
        }
        if ((b + 1) % kFoldBoxes == 0 || b + 1 == nb) {
#pragma unroll
          for (int k = 0; k < K; ++k) {
            fold_two_sum(H[k], L[k], acc[k]);
            acc[k] = 0.f;
          }
        }
        rh = nh;
        rl = nl;
      }
      float2* out = part + S.part + (long long)it.z * n;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const int i = g0 + k * 32 + lane;
        if (i < tb1) out[i] = make_float2(H[k], L[k]);
      }
    }
    if (sym) {
      // the transposed terms of the chunk's charges: the block's slot of their kind (the Kelvin
      // sums scaled by 1 / |x_j|, stored with the Kelvin record)
      __syncwarp();
      float2* out = part + S.part + (long long)(ch.type == 0 ? blk : S.ncr + blk) * n + ch.first;
      for (int j = lane; j < ch.count; j += 32) {
        float2 p = P[j];
        if (ch.type == 1) {
          const float w = __ldg(gl + j).w;
          p.x *= w;
          p.y *= w;
        }
        out[j] = p;
      }
      __syncwarp();
    }
  }
}
