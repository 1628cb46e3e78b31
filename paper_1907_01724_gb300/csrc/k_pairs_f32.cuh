// FP32 pair-sum kernel (included by k_pairs.cu inside namespace hsma).
//
// Sources and targets are in the spatial order of k_order.cu.  A warp owns 32*K consecutive
// targets, whose hi coordinates span a small box; every 32-source box of a staged tile is
// tested against it.  Boxes farther apart than sqrt(dc2) = kNearRel a take the plain FP32 form
//   r^2 = |x_hi - y_hi|^2        (3 FADD, 1 FMUL, 2 FFMA, then MUFU rsqrt and 1 FFMA per pair)
// whose error from rounding the coordinates to FP32 is at most ~2^-24 |x| / d relative per
// pair (d >= kNearRel a) and of random sign over the far sources; nearer boxes take the hi/lo
// form s = (x_hi - y_hi) + (x_lo - y_lo), r^2 = |s|^2, accurate to FP32 rounding at any
// distance (a charge next to its own Kelvin image).  The decision is uniform over the warp.
template <int NT, int K>
__global__ __launch_bounds__(NT) void k_pairs_f32(const SysDev* __restrict__ sys, PairWork w1, PairWork w2,
                                                  const float4* __restrict__ src_hi,
                                                  const float4* __restrict__ src_lo,
                                                  const float4* __restrict__ surf_a,
                                                  const float4* __restrict__ surf_b,
                                                  const float4* __restrict__ boxes, float2* __restrict__ part)
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
    const int w0 = t0 + warp * 32 * K;  // the warp's targets are [w0, w0 + 32 K)
    const ChunkInfo ch = decode_chunk(S, it.z);

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

    // targets (a slot past the end repeats the block's first target)
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
    // box of the warp's targets
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
    float H[K], L[K];
#pragma unroll
    for (int k = 0; k < K; ++k) H[k] = L[k] = 0.f;

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
      if (ch.type == 2) {
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
      } else {
        const int sbase = ch.first + t * NT;
        for (int u = 0; u < cnt; u += kBox) {
          const int ue = min(cnt, u + kBox);
          const long long bi = box_kind + (sbase + u) / kBox;
          const float4 bmn = __ldg(&boxes[2 * bi]), bmx = __ldg(&boxes[2 * bi + 1]);
          const float gx = fmaxf(0.f, fmaxf(wmnx - bmx.x, bmn.x - wmxx));
          const float gy = fmaxf(0.f, fmaxf(wmny - bmx.y, bmn.y - wmxy));
          const float gz = fmaxf(0.f, fmaxf(wmnz - bmx.z, bmn.z - wmxz));
          if (gx * gx + gy * gy + gz * gz > S.dc2) {
#pragma unroll 4
            for (int s = u; s < ue; ++s) {
              const float4 h = A[s];
#pragma unroll
              for (int k = 0; k < K; ++k) {
                const float dx = txh[k] - h.x, dy = tyh[k] - h.y, dz = tzh[k] - h.z;
                float r2 = dx * dx;
                r2 = fmaf(dy, dy, r2);
                r2 = fmaf(dz, dz, r2);
                acc[k] = fmaf(h.w, rsqrt_mufu(r2), acc[k]);
              }
            }
          } else if (ch.type == 0 && sbase + u < w0 + 32 * K && w0 < sbase + ue) {
            // the warp's own targets are among these sources: skip the self pair
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
                inv = (sbase + s == tix[k]) ? 0.f : inv;
                acc[k] = fmaf(h.w, inv, acc[k]);
              }
            }
          } else {
#pragma unroll 2
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
                acc[k] = fmaf(h.w, rsqrt_mufu(r2), acc[k]);
              }
            }
          }
        }
      }
      // two-sum fold of the tile partial
#pragma unroll
      for (int k = 0; k < K; ++k) {
        const float s = H[k] + acc[k];
        const float bp = s - H[k];
        L[k] += (H[k] - (s - bp)) + (acc[k] - bp);
        H[k] = s;
      }
      __syncthreads();
    }
    float2* out = part + S.part + (long long)it.z * n;
#pragma unroll
    for (int k = 0; k < K; ++k)
      if (tix[k] < n) out[tix[k]] = make_float2(H[k], L[k]);
  }
}
