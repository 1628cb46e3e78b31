// Treecode far field of the real-charge and Kelvin-image pair sums of one large cavity (FP32
// path).  The paper evaluates the pair sum of eq. phirffinall with the FMM for N up to 1e6
// (Sec. 4.2, Algorithm 1 step 5); here a GPU treecode over the records' Morton order replaces the
// direct real and Kelvin pair sums, and the surface images keep their direct sum (3M sources per
// target).
//
// Octree.  Node (l, c) is Morton cell c of the 2^l-per-axis grid over [-a, a]^3; its records are
// a contiguous run of sorted positions (k_order_keys / k_order_sort sort by a key of key_lv >= L
// levels).  The real tree's node holds the charges of the run, the Kelvin tree's node the images
// of the same charges, except images farther than kFarImageRel a from the centre ("far images"),
// which form one expansion about the centre instead.
//   k_tree_marks  record range of every node of levels kTreeTop..L (first and last position of
//                 each key prefix)
//   k_tree_leaf   level L: bounding box, centre, radius and the multipole moments of both trees
//                 (a warp per node, lane-strided records, fixed-order warp sums)
//   k_tree_up     levels L-1..kTreeTop: box and radius from the children, moments by shifting
//                 the children's moments to the parent's centre (a warp per node)
//   k_tree_far    the far images' expansion about the centre (fixed-order block sums, the last
//                 block adds the blocks in order)
//   k_tree_eval   persistent warps over items (32 consecutive targets, one tree, an eighth of
//                 its root cells): depth-first traversal of the item's subtrees from the
//                 level-kTreeTop cells; a node far from every target of the group (radius <=
//                 theta (distance of the target from the centre)) with at
//                 least cmin records is evaluated from its moments at each target, a near leaf (or a
//                 far node too small for its moments to pay) by the direct pair sum with hi/lo
//                 coordinate differences; then the far-image expansion at each target.  Writes the
//                 real and the Kelvin sums as the (hi, lo) partials of chunks 0..kTreeRootSplit-1
//                 and kTreeRootSplit..2 kTreeRootSplit-1, which the reduction adds as it adds every
//                 chunk.
// Every sum runs in a fixed order (no atomics on values), so results do not depend on scheduling.
//
// Solid harmonics (unnormalised associated Legendre functions P_n^m without the Condon-Shortley
// phase), for 0 <= m <= n:
//   R_n^m(x) = |x|^n P_n^m(cos t) e^{i m f} / (n + m)!,   I_n^m(x) = (n - m)! P_n^m(cos t) e^{i m f} / |x|^(n+1),
// so that, by the addition theorem of the Legendre polynomials, for |y| < |x|
//   1/|x - y| = sum_n [ R_n^0(y) I_n^0(x) + 2 Re sum_{m >= 1} conj(R_n^m(y)) I_n^m(x) ].
// Both satisfy three-term recurrences in Cartesian coordinates (r^2 = |x|^2):
//   R_m^m = R_{m-1}^{m-1} (x + i y) / (2m),     R_n^m = [(2n-1) z R_{n-1}^m - r^2 R_{n-2}^m] / (n^2 - m^2),
//   I_m^m = I_{m-1}^{m-1} (2m-1)(x + i y) / r^2, I_n^m = [(2n-1) z I_{n-1}^m - ((n-1)^2 - m^2) I_{n-2}^m] / r^2,
// with R_0^0 = 1, I_0^0 = 1/r.  A node of centre c and radius rho stores the moments
// M_n^m = sum_j Q_j conj(R_n^m((y_j - c)/rho)) and gives phi(x) = (1/rho) sum w_m Re(M_n^m I_n^m((x - c)/rho))
// (w_0 = 1, w_m = 2).  The far images give L_n^m = sum_j Q_j conj(I_n^m(y_j/a)) and
// phi(x) = (1/a) sum w_m Re(L_n^m R_n^m(x/a)) inside the cavity.
// Shift of a child's moments (centre c', radius rho') to the parent (c, rho): with b = (c' - c)/rho,
// s = rho'/rho, and the solid harmonics continued to m < 0 in the Condon-Shortley convention
// (X_n^{-m} = conj(X_n^m), X_n^m -> (-1)^m X_n^m for m > 0), the addition theorem
// R_n^m(u + v) = sum_{j,k} R_j^k(u) R_{n-j}^{m-k}(v) of the regular harmonics gives
//   M_n^m = (-1)^m sum_{j <= n} s^j sum_k A_j^k conj(B_{n-j}^{m-k}),
//   A_j^k = (-1)^k M'_j^k (k >= 0), conj(M'_j^{-k}) (k < 0);  B_l^t = (-1)^t R_l^t(b) (t >= 0), conj(R_l^{-t}(b)) (t < 0).
// Moments are stored by column: (n, m) at m (P + 1) - m (m - 1)/2 + (n - m).
#include <algorithm>
#include <cmath>

#include "df64.cuh"
#include "fp32_pair.cuh"
#include "tree.h"

namespace hsma {

__host__ __device__ constexpr int tree_col(int P, int m) { return m * (P + 1) - m * (m - 1) / 2; }

// Whether a Kelvin record lies beyond kFarImageRel a (its high part, rounded without contraction,
// so that every kernel classifies a record the same way).
__device__ __forceinline__ bool far_image(float4 h, float rfar2)
{
  return __fadd_rn(__fadd_rn(__fmul_rn(h.x, h.x), __fmul_rn(h.y, h.y)), __fmul_rn(h.z, h.z)) > rfar2;
}

__device__ __forceinline__ float warp_min(float v)
{
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v)
{
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------------------
// Record ranges: sorted position i starts node (l, c) if the previous record's key prefix
// differs, and ends it if the next one's does.  node[] is zeroed before (empty nodes keep 0, 0).
__global__ __launch_bounds__(256) void k_tree_marks(TreeView t)
{
  const SysDev& S = t.sys[0];
  const int n = S.n;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const long long c0 = S.chg;
  const int k = t.key[c0 + t.perm[c0 + i]];
  const int kp = i > 0 ? t.key[c0 + t.perm[c0 + i - 1]] : -1;
  const int kn = i + 1 < n ? t.key[c0 + t.perm[c0 + i + 1]] : -1;
  for (int l = kTreeTop; l <= t.L; ++l) {
    const int sh = 3 * (t.key_lv - l);
    const int id = k >> sh;
    const long long g = tree_node_index(l, id);
    if (i == 0 || (kp >> sh) != id) t.node[g].x = i;
    if (i == n - 1 || (kn >> sh) != id) t.node[g].y = i + 1;
  }
}

// ---------------------------------------------------------------------------------------
// Leaves: geometry and moments of both trees, a warp per level-L node.
constexpr int kLeafWarps = 4;
template <int P>
__global__ __launch_bounds__(32 * kLeafWarps) void k_tree_leaf(TreeView t)
{
  constexpr int NM = tree_nm(P);
  const int lane = threadIdx.x & 31;
  const long long c = (long long)blockIdx.x * kLeafWarps + (threadIdx.x >> 5);
  if (c >= (1LL << (3 * t.L))) return;  // whole warps
  const SysDev& S = t.sys[0];
  const int n = S.n;
  const long long nodes = tree_node_count(t.L);
  const long long g = tree_node_index(t.L, c);
  const int2 be = t.node[g];
  const float a = 1.f / t.inv_a;
  for (int tr = 0; tr < 2; ++tr) {
    const float4* __restrict__ H = t.hi + S.src + (long long)tr * n;
    const float4* __restrict__ Lo = t.lo + S.src + (long long)tr * n;
    float mn0 = 3.0e38f, mn1 = 3.0e38f, mn2 = 3.0e38f, mx0 = -3.0e38f, mx1 = -3.0e38f, mx2 = -3.0e38f;
    for (int j = be.x + lane; j < be.y; j += 32) {
      const float4 h = H[j];
      if (tr == 1 && far_image(h, t.rfar2)) continue;
      mn0 = fminf(mn0, h.x);
      mn1 = fminf(mn1, h.y);
      mn2 = fminf(mn2, h.z);
      mx0 = fmaxf(mx0, h.x);
      mx1 = fmaxf(mx1, h.y);
      mx2 = fmaxf(mx2, h.z);
    }
    mn0 = warp_min(mn0);
    mn1 = warp_min(mn1);
    mn2 = warp_min(mn2);
    mx0 = warp_max(mx0);
    mx1 = warp_max(mx1);
    mx2 = warp_max(mx2);
    float4* geo = t.geo + (long long)tr * nodes + g;
    float4* bx = t.box + 2 * ((long long)tr * nodes + g);
    float2* M = t.mom + ((long long)tr * nodes + g) * NM;
    if (!(mn0 <= mx0)) {
      if (lane == 0) {
        *geo = make_float4(0.f, 0.f, 0.f, -1.f);
        bx[0] = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f);
        bx[1] = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.f);
      }
      for (int k = lane; k < NM; k += 32) M[k] = make_float2(0.f, 0.f);
      continue;
    }
    const float cx = 0.5f * (mn0 + mx0), cy = 0.5f * (mn1 + mx1), cz = 0.5f * (mn2 + mx2);
    float r2max = 0.f;
    for (int j = be.x + lane; j < be.y; j += 32) {
      const float4 h = H[j];
      if (tr == 1 && far_image(h, t.rfar2)) continue;
      const float dx = h.x - cx, dy = h.y - cy, dz = h.z - cz;
      r2max = fmaxf(r2max, dx * dx + dy * dy + dz * dz);
    }
    // (a margin for the rounding of the hi coordinates and of the distance)
    const float rho = sqrtf(warp_max(r2max)) * 1.000001f + 2e-7f * a + 1e-6f * a;
    if (lane == 0) {
      *geo = make_float4(cx, cy, cz, rho);
      bx[0] = make_float4(mn0, mn1, mn2, 0.f);
      bx[1] = make_float4(mx0, mx1, mx2, 0.f);
    }
    const float ir = 1.f / rho;
#pragma unroll
    for (int m = 0; m <= P; ++m) {
      float cr[P + 1], ci[P + 1];
#pragma unroll
      for (int k = 0; k <= P - m; ++k) cr[k] = ci[k] = 0.f;
      for (int j = be.x + lane; j < be.y; j += 32) {
        const float4 h = H[j];
        if (tr == 1 && far_image(h, t.rfar2)) continue;
        const float4 l = Lo[j];
        const float vx = ((h.x - cx) + l.x) * ir, vy = ((h.y - cy) + l.y) * ir, vz = ((h.z - cz) + l.z) * ir;
        const float r2 = vx * vx + vy * vy + vz * vz;
        float dr = h.w, di = 0.f;  // Q R_m^m
#pragma unroll
        for (int k = 1; k <= m; ++k) {
          const float s = 0.5f / (float)k;
          const float nr = (dr * vx - di * vy) * s;
          di = (dr * vy + di * vx) * s;
          dr = nr;
        }
        float p0r = 0.f, p0i = 0.f, p1r = dr, p1i = di;
        cr[0] += p1r;
        ci[0] -= p1i;
#pragma unroll
        for (int nn = m + 1; nn <= P; ++nn) {
          const float A = (float)(2 * nn - 1) * vz;
          const float inv = 1.f / (float)(nn * nn - m * m);
          const float qr = (A * p1r - r2 * p0r) * inv, qi = (A * p1i - r2 * p0i) * inv;
          cr[nn - m] += qr;
          ci[nn - m] -= qi;
          p0r = p1r;
          p0i = p1i;
          p1r = qr;
          p1i = qi;
        }
      }
#pragma unroll
      for (int k = 0; k <= P - m; ++k) {
        const float sr = warp_sum(cr[k]), si = warp_sum(ci[k]);
        if (lane == 0) M[tree_col(P, m) + k] = make_float2(sr, si);
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// Upward pass, level l < L: a warp per node, from its 8 children (level l + 1).
constexpr int kUpWarps = 4;
template <int P>
__device__ __forceinline__ void decode_nm(int idx, int& n, int& m)
{
  m = 0;
  while (m < P && idx >= tree_col(P, m + 1)) ++m;
  n = m + (idx - tree_col(P, m));
}

template <int P>
__global__ __launch_bounds__(32 * kUpWarps) void k_tree_up(TreeView t, int l)
{
  constexpr int NM = tree_nm(P);
  constexpr int OUT = (NM + 31) / 32;
  constexpr int KW = 2 * P + 1;  // k = -P..P
  // per warp, for the child being shifted: A[j][k] = s^j A_j^k and B[l][t] = conj(B_l^t), dense
  // over -P <= k, t <= P (entries with |k| > j or |t| > l are never read)
  __shared__ float2 sAd[kUpWarps][(P + 1) * KW], sBd[kUpWarps][(P + 1) * KW];
  __shared__ float sPow[kUpWarps][P + 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long c = (long long)blockIdx.x * kUpWarps + w;
  if (c >= (1LL << (3 * l))) return;  // whole warps
  const long long nodes = tree_node_count(t.L);
  const long long g = tree_node_index(l, c);
  const long long g0 = tree_node_index(l + 1, 8 * c);
  int on[OUT], om[OUT];
#pragma unroll
  for (int q = 0; q < OUT; ++q) {
    const int idx = lane + 32 * q;
    if (idx < NM) {
      decode_nm<P>(idx, on[q], om[q]);
    } else {
      on[q] = -1;
      om[q] = 0;
    }
  }
  for (int tr = 0; tr < 2; ++tr) {
    const long long base = (long long)tr * nodes;
    float4 cg = make_float4(0.f, 0.f, 0.f, -1.f);
    float4 bmn = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f), bmx = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.f);
    if (lane < 8) {
      cg = t.geo[base + g0 + lane];
      if (cg.w >= 0.f) {
        bmn = t.box[2 * (base + g0 + lane)];
        bmx = t.box[2 * (base + g0 + lane) + 1];
      }
    }
    const bool ne = lane < 8 && cg.w >= 0.f;
    const unsigned any = __ballot_sync(0xffffffffu, ne);
    float4* geo = t.geo + base + g;
    float4* bx = t.box + 2 * (base + g);
    float2* M = t.mom + (base + g) * NM;
    if (!any) {
      if (lane == 0) {
        *geo = make_float4(0.f, 0.f, 0.f, -1.f);
        bx[0] = make_float4(3.0e38f, 3.0e38f, 3.0e38f, 0.f);
        bx[1] = make_float4(-3.0e38f, -3.0e38f, -3.0e38f, 0.f);
      }
      for (int k = lane; k < NM; k += 32) M[k] = make_float2(0.f, 0.f);
      continue;
    }
    const float mn0 = warp_min(bmn.x), mn1 = warp_min(bmn.y), mn2 = warp_min(bmn.z);
    const float mx0 = warp_max(bmx.x), mx1 = warp_max(bmx.y), mx2 = warp_max(bmx.z);
    const float cx = 0.5f * (mn0 + mx0), cy = 0.5f * (mn1 + mx1), cz = 0.5f * (mn2 + mx2);
    float rr = 0.f;
    if (ne) {
      const float dx = cg.x - cx, dy = cg.y - cy, dz = cg.z - cz;
      rr = sqrtf(dx * dx + dy * dy + dz * dz) + cg.w;
    }
    const float rho = warp_max(rr) * 1.000001f;
    if (lane == 0) {
      *geo = make_float4(cx, cy, cz, rho);
      bx[0] = make_float4(mn0, mn1, mn2, 0.f);
      bx[1] = make_float4(mx0, mx1, mx2, 0.f);
    }
    const float irp = 1.f / rho;
    float accr[OUT], acci[OUT];
#pragma unroll
    for (int q = 0; q < OUT; ++q) accr[q] = acci[q] = 0.f;
    for (int k = 0; k < 8; ++k) {
      if (!((any >> k) & 1u)) continue;  // uniform
      const float kx = __shfl_sync(0xffffffffu, cg.x, k), ky = __shfl_sync(0xffffffffu, cg.y, k);
      const float kz = __shfl_sync(0xffffffffu, cg.z, k), kr = __shfl_sync(0xffffffffu, cg.w, k);
      const float s = kr * irp;
      const float bxv = (kx - cx) * irp, byv = (ky - cy) * irp, bzv = (kz - cz) * irp;
      const float2* Mc = t.mom + (base + g0 + k) * NM;
      if (lane <= P) {
        // column m = lane of R(b) into B (both signs of t), and s^lane
        const int m = lane;
        const float r2 = bxv * bxv + byv * byv + bzv * bzv;
        float dr = 1.f, di = 0.f;
        for (int j = 1; j <= m; ++j) {
          const float f = 0.5f / (float)j;
          const float nr = (dr * bxv - di * byv) * f;
          di = (dr * byv + di * bxv) * f;
          dr = nr;
        }
        const float sgn = (m & 1) ? -1.f : 1.f;
        float p0r = 0.f, p0i = 0.f, p1r = dr, p1i = di;
        for (int nn = m; nn <= P; ++nn) {
          if (nn > m) {
            const float A = (float)(2 * nn - 1) * bzv;
            const float inv = 1.f / (float)(nn * nn - m * m);
            const float qr = (A * p1r - r2 * p0r) * inv, qi = (A * p1i - r2 * p0i) * inv;
            p0r = p1r;
            p0i = p1i;
            p1r = qr;
            p1i = qi;
          }
          // conj(B_nn^m) = (-1)^m conj(R_nn^m); conj(B_nn^-m) = R_nn^m
          sBd[w][nn * KW + P + m] = make_float2(sgn * p1r, -sgn * p1i);
          if (m > 0) sBd[w][nn * KW + P - m] = make_float2(p1r, p1i);
        }
        float sp = 1.f;
        for (int j = 0; j < m; ++j) sp *= s;
        sPow[w][m] = sp;
      }
      __syncwarp();
      for (int e = lane; e < (P + 1) * KW; e += 32) {
        const int j = e / KW, kk = e - j * KW - P;
        if (kk > j || -kk > j) continue;
        const int ka = kk >= 0 ? kk : -kk;
        float2 A = Mc[tree_col(P, ka) + j - ka];
        if (kk >= 0) {
          if (kk & 1) A = make_float2(-A.x, -A.y);
        } else {
          A.y = -A.y;
        }
        const float sj = sPow[w][j];
        sAd[w][e] = make_float2(sj * A.x, sj * A.y);
      }
      __syncwarp();
#pragma unroll
      for (int q = 0; q < OUT; ++q) {
        const int n = on[q], m = om[q];
        if (n < 0) continue;
        float ar = 0.f, ai = 0.f;
        for (int j = 0; j <= n; ++j) {
          const int l2 = n - j;
          const int k0 = max(-j, m - l2), k1 = min(j, m + l2);
          const float2* Aj = &sAd[w][j * KW + P];
          const float2* Bl = &sBd[w][l2 * KW + P + m];  // Bl[-kk] = conj(B_{l2}^{m-kk})
          for (int kk = k0; kk <= k1; ++kk) {
            const float2 A = Aj[kk], B = Bl[-kk];
            ar = fmaf(A.x, B.x, ar);
            ar = fmaf(-A.y, B.y, ar);
            ai = fmaf(A.x, B.y, ai);
            ai = fmaf(A.y, B.x, ai);
          }
        }
        accr[q] += ar;
        acci[q] += ai;
      }
      __syncwarp();
    }
#pragma unroll
    for (int q = 0; q < OUT; ++q) {
      if (on[q] < 0) continue;
      const float sg = (om[q] & 1) ? -1.f : 1.f;
      M[lane + 32 * q] = make_float2(sg * accr[q], sg * acci[q]);
    }
  }
}

// ---------------------------------------------------------------------------------------
// Far images: L_n^m = sum Q conj(I_n^m(y/a)) over Kelvin records beyond kFarImageRel a.
constexpr int kFarWarps = 8;
constexpr int kFarNM = tree_nm(kFarOrder);
__global__ __launch_bounds__(32 * kFarWarps) void k_tree_far(TreeView t)
{
  __shared__ float2 acc[kFarWarps][kFarNM];
  __shared__ bool last;
  const SysDev& S = t.sys[0];
  const int n = S.n;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kFarWarps * kFarNM; i += blockDim.x) (&acc[0][0])[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const int per = ((n + kFarBlocks - 1) / kFarBlocks + 31) / 32 * 32;
  const int r0 = blockIdx.x * per, r1 = min(n, r0 + per);
  for (int j0 = r0 + 32 * w; j0 < r1; j0 += 32 * kFarWarps) {
    const int j = j0 + lane;
    float4 h = make_float4(0.f, 0.f, 0.f, 0.f), lo = h;
    bool far = false;
    if (j < r1) {
      h = t.hi[S.src + n + j];
      far = far_image(h, t.rfar2);
      if (far) lo = t.lo[S.src + n + j];
    }
    if (!__any_sync(0xffffffffu, far)) continue;
    // other lanes evaluate a dummy point 4a out on the x axis with zero strength
    const float Q = far ? h.w : 0.f;
    const float ux = far ? (h.x + lo.x) * t.inv_a : 4.f, uy = far ? (h.y + lo.y) * t.inv_a : 0.f;
    const float uz = far ? (h.z + lo.z) * t.inv_a : 0.f;
    const float r2 = ux * ux + uy * uy + uz * uz;
    const float i2 = __frcp_rn(r2);
    float dr = Q * rsqrt_mufu(r2), di = 0.f;  // Q I_0^0
#pragma unroll
    for (int m = 0; m <= kFarOrder; ++m) {
      if (m > 0) {
        const float f = (float)(2 * m - 1) * i2;
        const float nr = (dr * ux - di * uy) * f;
        di = (dr * uy + di * ux) * f;
        dr = nr;
      }
      float cr[kFarOrder + 1], ci[kFarOrder + 1];
      float p0r = 0.f, p0i = 0.f, p1r = dr, p1i = di;
      cr[0] = p1r;
      ci[0] = -p1i;
#pragma unroll
      for (int nn = m + 1; nn <= kFarOrder; ++nn) {
        const float A = (float)(2 * nn - 1) * uz, B = (float)((nn - 1) * (nn - 1) - m * m);
        const float qr = (A * p1r - B * p0r) * i2, qi = (A * p1i - B * p0i) * i2;
        cr[nn - m] = qr;
        ci[nn - m] = -qi;
        p0r = p1r;
        p0i = p1i;
        p1r = qr;
        p1i = qi;
      }
#pragma unroll
      for (int k = 0; k <= kFarOrder - m; ++k) {
        const float sr = warp_sum(cr[k]), si = warp_sum(ci[k]);
        if (lane == 0) {
          float2& a = acc[w][tree_col(kFarOrder, m) + k];
          a.x += sr;
          a.y += si;
        }
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kFarNM; i += blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
#pragma unroll
    for (int q = 0; q < kFarWarps; ++q) {
      s.x += acc[q][i].x;
      s.y += acc[q][i].y;
    }
    t.farp[(long long)blockIdx.x * kFarNM + i] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(t.ctr, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int i = threadIdx.x; i < kFarNM; i += blockDim.x) {
    float2 s = make_float2(0.f, 0.f);
    for (int b = 0; b < (int)gridDim.x; ++b) {
      const float2 v = __ldcg(t.farp + (long long)b * kFarNM + i);
      s.x += v.x;
      s.y += v.y;
    }
    t.farL[i] = s;
  }
  if (threadIdx.x == 0) *t.ctr = 0u;
}

// ---------------------------------------------------------------------------------------
// Evaluation.
// phi at target (th, tl) of a node's moments M (stored to order P; centre and radius gc), the
// series truncated at order Q <= P.
template <int P, int Q>
__device__ __forceinline__ float m2p(const float2* __restrict__ M, float4 gc, float4 th, float4 tl)
{
  const float ir = 1.f / gc.w;
  const float ux = ((th.x - gc.x) + tl.x) * ir, uy = ((th.y - gc.y) + tl.y) * ir, uz = ((th.z - gc.z) + tl.z) * ir;
  const float r2 = ux * ux + uy * uy + uz * uz;
  const float i2 = __frcp_rn(r2);
  const float px = ux * i2, py = uy * i2, wz = uz * i2;
  float dr = rsqrt_mufu(r2), di = 0.f;  // I_0^0
  float acc = 0.f;
  {
    // m = 0: the column is real (written out: IEEE arithmetic does not let the compiler drop
    // the zero imaginary parts)
    float p0 = 0.f, p1 = dr;
    float col = __ldg(M).x * dr;
#pragma unroll
    for (int nn = 1; nn <= Q; ++nn) {
      const float A = (float)(2 * nn - 1) * wz, B = (float)((nn - 1) * (nn - 1)) * i2;
      const float q = A * p1 - B * p0;
      col = fmaf(__ldg(M + nn).x, q, col);
      p0 = p1;
      p1 = q;
    }
    acc = col;
  }
#pragma unroll
  for (int m = 1; m <= Q; ++m) {
    {
      const float f = (float)(2 * m - 1);
      const float nr = f * (dr * px - di * py);
      di = f * (dr * py + di * px);
      dr = nr;
    }
    const float2* Mc = M + tree_col(P, m);
    float2 mm = __ldg(Mc);
    float col = mm.x * dr - mm.y * di;
    float p0r = 0.f, p0i = 0.f, p1r = dr, p1i = di;
#pragma unroll
    for (int nn = m + 1; nn <= Q; ++nn) {
      const float A = (float)(2 * nn - 1) * wz, B = (float)((nn - 1) * (nn - 1) - m * m) * i2;
      const float qr = A * p1r - B * p0r, qi = A * p1i - B * p0i;
      mm = __ldg(Mc + (nn - m));
      col = fmaf(mm.x, qr, col);
      col = fmaf(-mm.y, qi, col);
      p0r = p1r;
      p0i = p1i;
      p1r = qr;
      p1i = qi;
    }
    acc = fmaf(2.f, col, acc);
  }
  return acc * ir;
}

// The same sum row by row (n outer), truncated at a runtime order q <= P: rows n and n - 1 of
// I_n^m stay in registers, so one code path serves every order (the nodes far beyond the opening
// criterion need far fewer terms for the same truncation bound).
template <int P>
__device__ __forceinline__ float m2p_rows(const float2* M, float4 gc, float4 th, float4 tl, int q)
{
  const float ir = 1.f / gc.w;
  const float ux = ((th.x - gc.x) + tl.x) * ir, uy = ((th.y - gc.y) + tl.y) * ir, uz = ((th.z - gc.z) + tl.z) * ir;
  const float r2 = ux * ux + uy * uy + uz * uz;
  const float i2 = __frcp_rn(r2);
  const float px = ux * i2, py = uy * i2, wz = uz * i2;
  // rows n - 1 (a) and n - 2 (b) as (re, im) pairs: the recurrence's complex-by-real products
  // and the dot product with the (re, -im) moments as packed FP32 (FFMA2 / FMUL2)
  float2 a[P + 1], b[P + 1];
#pragma unroll
  for (int m = 0; m <= P; ++m) a[m] = b[m] = make_float2(0.f, 0.f);
  a[0].x = rsqrt_mufu(r2);  // I_0^0
  float acc0 = M[0].x * a[0].x;       // m = 0 terms
  float2 acc1 = make_float2(0.f, 0.f);  // m > 0 terms (weight 2): the re re and -im im parts
#pragma unroll
  for (int n = 1; n <= P; ++n) {
    if (n > q) break;
    const float A = (float)(2 * n - 1) * wz;
    const float2 A2 = make_float2(A, A);
    // the new diagonal I_n^n from I_{n-1}^{n-1}
    const float f = (float)(2 * n - 1);
    const float dr = f * (a[n - 1].x * px - a[n - 1].y * py), di = f * (a[n - 1].x * py + a[n - 1].y * px);
#pragma unroll
    for (int m = 0; m < n; ++m) {
      const float nB = (float)(m * m - (n - 1) * (n - 1)) * i2;  // -B (zero for m = n - 1)
      const float2 nv = __ffma2_rn(make_float2(nB, nB), b[m], __fmul2_rn(A2, a[m]));
      b[m] = a[m];
      a[m] = nv;
      const float2 mm = M[tree_col(P, m) + (n - m)];
      if (m == 0)
        acc0 = fmaf(mm.x, nv.x, acc0);
      else
        acc1 = __ffma2_rn(mm, nv, acc1);
    }
    b[n] = make_float2(0.f, 0.f);
    a[n] = make_float2(dr, di);
    acc1 = __ffma2_rn(M[tree_col(P, n)], a[n], acc1);
  }
  return fmaf(2.f, acc1.x + acc1.y, acc0) * ir;
}

// phi at the target of the far images' expansion (|x| < a)
__device__ __forceinline__ float l2p_far(const float2* __restrict__ L, float4 th, float4 tl, float inv_a)
{
  const float ux = (th.x + tl.x) * inv_a, uy = (th.y + tl.y) * inv_a, uz = (th.z + tl.z) * inv_a;
  const float r2 = ux * ux + uy * uy + uz * uz;
  float dr = 1.f, di = 0.f;  // R_0^0
  float acc = 0.f;
  // (once per Kelvin item: rolled loops keep the registers for the traversal)
#pragma unroll 1
  for (int m = 0; m <= kFarOrder; ++m) {
    if (m > 0) {
      const float f = 0.5f / (float)m;
      const float nr = (dr * ux - di * uy) * f;
      di = (dr * uy + di * ux) * f;
      dr = nr;
    }
    const float2* Lc = L + tree_col(kFarOrder, m);
    float2 ll = __ldg(Lc);
    float col = ll.x * dr - ll.y * di;
    float p0r = 0.f, p0i = 0.f, p1r = dr, p1i = di;
#pragma unroll 1
    for (int nn = m + 1; nn <= kFarOrder; ++nn) {
      const float A = (float)(2 * nn - 1) * uz;
      const float inv = 1.f / (float)(nn * nn - m * m);
      const float qr = (A * p1r - r2 * p0r) * inv, qi = (A * p1i - r2 * p0i) * inv;
      ll = __ldg(Lc + (nn - m));
      col = fmaf(ll.x, qr, col);
      col = fmaf(-ll.y, qi, col);
      p0r = p1r;
      p0i = p1i;
      p1r = qr;
      p1i = qi;
    }
    acc += m == 0 ? col : 2.f * col;
  }
  return acc * inv_a;
}

// Direct sum of the records [be.x, be.y) at the lane's target, staged 32 at a time through the
// warp's shared buffers, with the exact (hi, lo) coordinate difference of inv_hilo (accurate to
// FP32 rounding at any distance, e.g. a charge next to its own Kelvin image).  checked: the node
// holds some of the group's own targets, and the source at sorted position `self` is skipped;
// kelvin: records beyond rfar2 count as zero.  Each batch's FP32 sum is added to the compensated
// total (a leaf of a dense cluster holds thousands of sources of similar size and mixed sign).
__device__ __forceinline__ void p2p(const float4* __restrict__ H, const float4* __restrict__ Lo, int2 be, float4 th,
                                    float4 tl, int self, bool checked, bool kelvin, float rfar2, float4* sh, float4* sl,
                                    df& total)
{
  const int lane = threadIdx.x & 31;
  for (int j0 = be.x; j0 < be.y; j0 += 32) {
    float acc = 0.f;  // one batch of 32 sources, folded into the compensated total below
    const int j = j0 + lane;
    __syncwarp();  // the previous batch has been read
    if (j < be.y) {
      float4 h = H[j];
      if (kelvin && far_image(h, rfar2)) h.w = 0.f;
      sh[lane] = h;
      sl[lane] = Lo[j];
    }
    __syncwarp();
    const int m = min(32, be.y - j0);
    if (!checked) {
#pragma unroll 4
      for (int k = 0; k < m; ++k) {
        const float4 s = sh[k], u = sl[k];
        acc = fmaf(s.w, inv_hilo(th.x, th.y, th.z, tl.x, tl.y, tl.z, s.x, s.y, s.z, u.x, u.y, u.z), acc);
      }
    } else {
      for (int k = 0; k < m; ++k) {
        const float4 s = sh[k], u = sl[k];
        const float v = s.w * inv_hilo(th.x, th.y, th.z, tl.x, tl.y, tl.z, s.x, s.y, s.z, u.x, u.y, u.z);
        acc += (j0 + k == self) ? 0.f : v;
      }
    }
    total = total + two_sum(acc, 0.f);
  }
}

// One work item: a group of 32 consecutive targets (sorted positions 32 grp ..) against the
// subtrees of one tree below root cells [rs R/kTreeRootSplit, (rs + 1) R/kTreeRootSplit) (tr = 0:
// real charges, 1: Kelvin images, the far-image expansion with rs = 0); traversal and evaluation,
// written to the item's own partial row (chunk tr kTreeRootSplit + rs).
template <int P>
__device__ __forceinline__ void eval_group(const TreeView& t, float2* __restrict__ part, int grp, int tr, int rs,
                                           int* stk, int2* sbe, float4* sgc, float4* sh, float4* sl, float2* smom)
{
  constexpr int NM = tree_nm(P);
  const int lane = threadIdx.x & 31;
  const SysDev& S = t.sys[0];
  const int n = S.n;
  const int i = grp * 32 + lane;
  const bool on = i < n;
  const int ic = on ? i : n - 1;
  const float4 th = t.hi[S.src + ic], tl = t.lo[S.src + ic];
  const float theta2 = t.theta * t.theta, margin = 4e-7f / t.inv_a;
  const long long nodes = tree_node_count(t.L);
  df acc = df_make(0.f, 0.f);
  constexpr int R = 1 << (3 * kTreeTop);
  {
    const float4* __restrict__ H = t.hi + S.src + (long long)tr * n;
    const float4* __restrict__ Lo = t.lo + S.src + (long long)tr * n;
    const float4* __restrict__ G = t.geo + (long long)tr * nodes;
    const float2* __restrict__ MM = t.mom + (long long)tr * nodes * NM;
    const int self = tr == 0 ? i : -1;
    __syncwarp();
    constexpr int RS = R / kTreeRootSplit;
    static_assert(RS <= 32, "a lane per root of an item");
    // depth first: an opened node leaves at most 8 - 1 more entries, once per level below the roots
    static_assert(RS + 7 * (kTreeMaxLevel - kTreeTop) <= kTreeStack, "traversal stack depth");
    int sp = 0;
    {
      // the item's roots with sources, the lowest cell on top; a stack entry carries the node's
      // record range and geometry, read when it is pushed (eight or fewer loads side by side)
      const long long gr = tree_node_index(kTreeTop, rs * RS + lane);
      int2 rb = make_int2(0, 0);
      float4 rgc = make_float4(0.f, 0.f, 0.f, -1.f);
      if (lane < RS) {
        rb = t.node[gr];
        if (rb.y > rb.x) rgc = G[gr];
      }
      const unsigned ok = __ballot_sync(0xffffffffu, lane < RS && rb.y > rb.x && rgc.w >= 0.f);
      if (lane < RS && ((ok >> lane) & 1u)) {
        const int at = __popc(ok >> (lane + 1));
        stk[at] = (kTreeTop << 26) | (rs * RS + lane);
        sbe[at] = rb;
        sgc[at] = rgc;
      }
      sp = __popc(ok);
      __syncwarp();
    }
    while (sp > 0) {
      --sp;
      const int e = stk[sp];
      const int2 be = sbe[sp];
      const float4 gc = sgc[sp];
      __syncwarp();  // every lane has read the entry before a push overwrites it
      const int l = e >> 26, c = e & ((1 << 26) - 1);
      const long long g = tree_node_index(l, c);
      // the node is far when its series converges with ratio rho / |t - c| <= theta at every
      // target of the group (each lane tests its own target; a margin covers the lo parts)
      const float dx = th.x - gc.x, dy = th.y - gc.y, dz = th.z - gc.z;
      const float rm = gc.w + margin;
      const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
      const bool far = __all_sync(0xffffffffu, rm * rm <= theta2 * d2);
      if (far && be.y - be.x >= t.cmin) {
        // the order whose truncation at the group's largest ratio rho/|t - c| stays within a tenth
        // of the order-P bound at theta: (q + 1) log(ratio) <= log(0.1 theta^(P+1))
        if constexpr (P <= 12) {
          const float r2max = warp_max(rm * rm / d2);
          const int q = min(P, max(2, (int)ceilf(t.log_eps / (0.5f * __logf(r2max))) - 1));
          // the node's moments staged in shared memory by one coalesced warp load
          const float2* src = MM + g * NM;
          for (int i = lane; i < NM; i += 32) {
            const float2 v = __ldg(src + i);
            smom[i] = make_float2(v.x, -v.y);  // (re, -im): the series' dot product as FFMA2
          }
          __syncwarp();
          acc = acc + two_sum(m2p_rows<P>(smom, gc, th, tl, q), 0.f);
          __syncwarp();
        } else {
          // (two rows of order 16 do not fit the registers: every node at order P, by columns)
          acc = acc + two_sum(m2p<P, P>(MM + g * NM, gc, th, tl), 0.f);
        }
      } else if (far || l == t.L) {
        const bool checked = tr == 0 && be.x < grp * 32 + 32 && be.y > grp * 32;
        p2p(H, Lo, be, th, tl, self, checked, tr == 1, t.rfar2, sh, sl, acc);
      } else {
        // open: the children with sources, the lowest cell on top
        const long long gch = tree_node_index(l + 1, 8LL * c);
        int2 cb = make_int2(0, 0);
        float4 cg = make_float4(0.f, 0.f, 0.f, -1.f);
        if (lane < 8) {
          cb = t.node[gch + lane];
          if (cb.y > cb.x) cg = G[gch + lane];
        }
        const unsigned ne = __ballot_sync(0xffffffffu, lane < 8 && cb.y > cb.x && cg.w >= 0.f);
        if (lane < 8 && ((ne >> lane) & 1u)) {
          const int at = sp + __popc(ne >> (lane + 1));
          stk[at] = ((l + 1) << 26) | (8 * c + lane);
          sbe[at] = cb;
          sgc[at] = cg;
        }
        sp += __popc(ne);
        __syncwarp();
      }
    }
  }
  if (tr == 1 && rs == 0) acc = acc + two_sum(l2p_far(t.farL, th, tl, t.inv_a), 0.f);
  if (on) part[S.part + (long long)(tr * kTreeRootSplit + rs) * n + i] = make_float2(acc.hi, acc.lo);
}

template <int P>
__global__ __launch_bounds__(32 * kTreeEvalWarps, kTreeEvalMinBlocks) void k_tree_eval(TreeView t,
                                                                                       float2* __restrict__ part)
{
  constexpr int NM = tree_nm(P);
  __shared__ int s_stack[kTreeEvalWarps][kTreeStack];
  __shared__ int2 s_sbe[kTreeEvalWarps][kTreeStack];
  __shared__ float4 s_sgc[kTreeEvalWarps][kTreeStack];
  __shared__ float2 s_mom[kTreeEvalWarps][NM];
  __shared__ float4 s_h[kTreeEvalWarps][32], s_l[kTreeEvalWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const SysDev& S = t.sys[0];
  const int n = S.n;
  constexpr int IPG = 2 * kTreeRootSplit;  // items per group
  const int items = IPG * ((n + 31) / 32), workers = gridDim.x * kTreeEvalWarps;
  // persistent warps: the first item by the warp's index, then items from the work counter (the
  // cost of an item varies with its distance from the interface and from the centre)
  for (int it = blockIdx.x * kTreeEvalWarps + w; it < items;) {
    const int r = it % IPG;
    eval_group<P>(t, part, it / IPG, r & 1, r >> 1, s_stack[w], s_sbe[w], s_sgc[w], s_h[w], s_l[w], s_mom[w]);
    int nx = 0;
    if (lane == 0) nx = workers + (int)atomicAdd(t.ctr + 1, 1u);
    it = __shfl_sync(0xffffffffu, nx, 0);
  }
}

// ---------------------------------------------------------------------------------------
int tree_levels(long long n)
{
  // leaves of ~25-50 charges for charges spread through the ball (52 % of the cube)
  const double v = std::log(std::max<double>((double)n, 1.0) / 25.0) / std::log(8.0);
  return std::min(kTreeMaxLevel, std::max(3, (int)std::lround(v)));
}

bool tree_order_supported(int P) { return P == 8 || P == 12 || P == 16; }

template <int P>
static void build_p(const TreeView& t, int n, cudaStream_t st)
{
  const long long leaves = 1LL << (3 * t.L);
  k_tree_leaf<P><<<(unsigned)((leaves + kLeafWarps - 1) / kLeafWarps), 32 * kLeafWarps, 0, st>>>(t);
  for (int l = t.L - 1; l >= kTreeTop; --l) {
    const long long cells = 1LL << (3 * l);
    k_tree_up<P><<<(unsigned)((cells + kUpWarps - 1) / kUpWarps), 32 * kUpWarps, 0, st>>>(t, l);
  }
}

void launch_tree_build(const TreeView& t, int n, cudaStream_t st)
{
  cudaMemsetAsync(t.node, 0, sizeof(int2) * (size_t)tree_node_count(t.L), st);
  cudaMemsetAsync(t.ctr, 0, 2 * sizeof(unsigned int), st);  // k_tree_far's and k_tree_eval's counters
  if (n <= 0) return;
  k_tree_marks<<<(n + 255) / 256, 256, 0, st>>>(t);
  if (t.P == 8) build_p<8>(t, n, st);
  else if (t.P == 12) build_p<12>(t, n, st);
  else build_p<16>(t, n, st);
  k_tree_far<<<kFarBlocks, 32 * kFarWarps, 0, st>>>(t);
}

void launch_tree_eval(const TreeView& t, int n, float2* part, cudaStream_t st)
{
  if (n <= 0) return;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  const int items = 2 * kTreeRootSplit * ((n + 31) / 32);
  const unsigned blocks = (unsigned)std::min<long long>((items + kTreeEvalWarps - 1) / kTreeEvalWarps,
                                                        (long long)sms * kTreeEvalMinBlocks);
  if (t.P == 8) k_tree_eval<8><<<blocks, 32 * kTreeEvalWarps, 0, st>>>(t, part);
  else if (t.P == 12) k_tree_eval<12><<<blocks, 32 * kTreeEvalWarps, 0, st>>>(t, part);
  else k_tree_eval<16><<<blocks, 32 * kTreeEvalWarps, 0, st>>>(t, part);
}

}  // namespace hsma
