// Direct tiled Coulomb sum of HSMA (Algorithm 1 step 5, eq. phirffinall of Fu & Gan,
// arXiv:1907.01724) and the FP64 reduction to potentials and energies.
//
// Sources of one cavity: n real charges (excluding the target itself), n trapezoid-modified
// Kelvin images, and M surface points each carrying a monopole and a dipole (the 3M discrete
// images of eq. phicorrfinall).  Work is split into items (system, target block, source
// chunk); persistent CTAs pull items from an atomic counter (longest items first) and write
// one compensated FP32 partial per (chunk, target), which k_reduce sums in a fixed order
// (FP64, or double-float on the FP32 path), so results do not depend on scheduling.  Records
// and partials are in the spatial order of k_order.cu; k_reduce maps them back to input order.
//
// FP32 path (ALU bound, no tensor cores: the sum is not a dense contraction):
//  * real and Kelvin records hold hi/lo-split coordinates; with dh the FP32 difference of the
//    high parts (exact for nearby points) and dl that of the low parts, s = dh + dl is the
//    coordinate difference to FP32 relative accuracy and r^2 = sum s^2, even for a charge next
//    to its own image (4 FP32 operations per coordinate); sources in a 32-record box farther
//    than kNearRel a from the box of a warp's targets use the hi parts alone (1 operation per
//    coordinate), see k_pairs_f32.cuh;
//  * 1/r is one MUFU rsqrt.approx per pair;
//  * each target keeps an FP32 partial per staged tile, folded into an (hi, lo) two-sum pair;
//  * surface points apply the dipole layer in its dy -> 0 limit sharing the monopole's rsqrt.
// FP64 path: the same structure in double precision with the central-difference dipole in
// the cancellation-free form 2 (R_tau - x.yhat) / (d+ d- (d+ + d-)).
#include <math.h>

#include "df64.cuh"
#include "hsma_internal.cuh"

namespace hsma {

__device__ __forceinline__ float rsqrt_mufu(float x)
{
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait()
{
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct ChunkInfo {
  int type;       // 0 real, 1 Kelvin, 2 surface
  int first;      // index of the first source within its kind
  int count;      // sources in the chunk
  long long off;  // record offset of the first source
};

__device__ __forceinline__ ChunkInfo decode_chunk(const SysDev& S, int c)
{
  ChunkInfo ci;
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

// ---------------------------------------------------------------------------------------
#include "k_pairs_f32.cuh"

// Tile configurations: kernel variants (CTA threads, targets per thread), each with 4, 2 or 1
// pair items per resident CTA slot (fewer, larger items have less per-item overhead, more items
// balance better); the autotuner picks one per size class.
#define HSMA_PAIR_CONFIGS(X) \
  X(0, 128, 4) X(1, 128, 2) X(2, 256, 2) X(3, 256, 4) X(4, 64, 4) X(5, 128, 1) X(6, 256, 1) X(7, 128, 8) \
  X(8, 64, 2) X(9, 64, 1) X(10, 32, 2) X(11, 32, 4)

static const int kPairKernel[][2] = {
#define HSMA_CFG_ENTRY(i, nt, k) {nt, k},
    HSMA_PAIR_CONFIGS(HSMA_CFG_ENTRY)
#undef HSMA_CFG_ENTRY
};
constexpr int kPairKernels = (int)(sizeof(kPairKernel) / sizeof(kPairKernel[0]));
static const int kItemsPerSlot[] = {4, 2, 1};
constexpr int kItemChoices = (int)(sizeof(kItemsPerSlot) / sizeof(kItemsPerSlot[0]));

int pair_config_count() { return kPairKernels * kItemChoices; }
int pair_kernel_of(int cfg) { return cfg % kPairKernels; }
PairConfig pair_config(int idx)
{
  PairConfig c;
  c.threads = kPairKernel[idx % kPairKernels][0];
  c.k = kPairKernel[idx % kPairKernels][1];
  c.items_per_slot = kItemsPerSlot[idx / kPairKernels];
  return c;
}

int pairs_f32_occupancy(int cfg)
{
  int b = 0;
  switch (pair_kernel_of(cfg)) {
#define HSMA_CFG_OCC(i, nt, k) \
  case i: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs_f32<nt, k>, nt, 0); break;
    HSMA_PAIR_CONFIGS(HSMA_CFG_OCC)
#undef HSMA_CFG_OCC
    default: break;
  }
  return b;
}

void launch_pairs_f32(int cfg, int grid, const SysDev* sys, PairWork w1, PairWork w2, const float4* src_hi,
                      const float4* src_lo, const float4* surf_a, const float4* surf_b, const float4* boxes,
                      float2* part, cudaStream_t st)
{
  switch (pair_kernel_of(cfg)) {
#define HSMA_CFG_LAUNCH(i, nt, k)                                                                          \
  case i:                                                                                                  \
    launch_k(k_pairs_f32<nt, k>, grid, nt, 0, st, false, sys, w1, w2, src_hi, src_lo, surf_a, surf_b, boxes, part); \
    break;
    HSMA_PAIR_CONFIGS(HSMA_CFG_LAUNCH)
#undef HSMA_CFG_LAUNCH
    default: break;
  }
}

// ---------------------------------------------------------------------------------------
// FP64 comparator path: one target per thread, plain staged loads.
constexpr int kF64Threads = kF64TargetsPerBlock;

__global__ __launch_bounds__(kF64Threads) void k_pairs_f64(const SysDev* __restrict__ sys, PairWork w1,
                                                           PairWork w2, const dbl4* __restrict__ src64,
                                                           const dbl4* __restrict__ surf64_a,
                                                           const double* __restrict__ surf64_b,
                                                           double* __restrict__ part64)
{
  __shared__ dbl4 shA[kF64Threads];
  __shared__ double shB[kF64Threads];
  __shared__ int s_item, s_list;
  const int tid = threadIdx.x;
  int list = 0;
  bool first_fetch = true;
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
    const int i = it.y * kF64Threads + tid;
    const dbl4 tg = src64[S.src + (i < n ? i : it.y * kF64Threads)];
    const ChunkInfo ch = decode_chunk(S, it.z);
    const double Rt = S.Rtau, rm = S.Rtau - 0.5 * S.dy, rp = S.Rtau + 0.5 * S.dy;
    double acc = 0.0;
    for (int t0 = 0; t0 < ch.count; t0 += kF64Threads) {
      const int cnt = min(kF64Threads, ch.count - t0);
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
          const double dx = tg.x - y.x, dy = tg.y - y.y, dz = tg.z - y.z;
          acc += y.w * rsqrt(dx * dx + dy * dy + dz * dz);
          const double rho = sqrt(y.x * y.x + y.y * y.y + y.z * y.z);
          const double hx = y.x / rho, hy = y.y / rho, hz = y.z / rho;
          const double mx = tg.x - rm * hx, my = tg.y - rm * hy, mz = tg.z - rm * hz;
          const double px = tg.x - rp * hx, py = tg.y - rp * hy, pz = tg.z - rp * hz;
          const double dm = sqrt(mx * mx + my * my + mz * mz);
          const double dp = sqrt(px * px + py * py + pz * pz);
          const double xy = tg.x * hx + tg.y * hy + tg.z * hz;
          acc += D * 2.0 * (Rt - xy) / (dp * dm * (dp + dm));
        }
      } else {
        const int sb = ch.first + t0;
        for (int s = 0; s < cnt; ++s) {
          const dbl4 h = shA[s];
          if (ch.type == 0 && sb + s == i) continue;
          // separately rounded IEEE operations and a correctly rounded sqrt and division: the
          // distance of a charge to its own nearby Kelvin image is ill-conditioned, so this path
          // evaluates it exactly as the plain definition does
          const double dx = tg.x - h.x, dy = tg.y - h.y, dz = tg.z - h.z;
          const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
          acc += h.w / sqrt(r2);
        }
      }
      __syncthreads();
    }
    if (i < n) part64[S.part + (long long)it.z * n + i] = acc;
  }
}

int pairs_f64_occupancy()
{
  int b = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs_f64, kF64Threads, 0);
  return b;
}

void launch_pairs_f64(int grid, const SysDev* sys, PairWork w1, PairWork w2, const dbl4* src64,
                      const dbl4* surf64_a, const double* surf64_b, double* part64, cudaStream_t st)
{
  launch_k(k_pairs_f64, grid, kF64Threads, 0, st, false, sys, w1, w2, src64, surf64_a, surf64_b, part64);
}

// ---------------------------------------------------------------------------------------
// phi_coul = sum of real-chunk partials, phi_rf = Kelvin + surface partials + centre constant,
// energies E_total = 1/2 sum q (phi_coul + phi_rf), E_RF = 1/2 sum q phi_rf.  Fixed-order
// block reductions; the last block of a system to finish (counter[r] per launch-local system
// r, reset by that block) sums the system's block partials in a fixed order.
constexpr int kRedLanes = 8;
// Sums of the (hi, lo) partials of this lane's chunks k = sub, sub + kRedLanes, ... < nch in
// ascending order: the real chunks (k < ncr) into c, the others into r.  Eight chunks' loads are
// issued ahead of their additions, so a target's partials cost one or two L2 round trips
// instead of one per chunk.
__device__ __forceinline__ void sum_chunks(const float2* __restrict__ b, long long n, int sub, int ncr, int nch,
                                           df& c, df& r)
{
  constexpr int kBatch = 8;
  for (int k0 = sub; k0 < nch; k0 += kBatch * 8) {
    float2 v[kBatch];
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      const int k = k0 + 8 * j;
      v[j] = k < nch ? b[(long long)k * n] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < kBatch; ++j) {
      const int k = k0 + 8 * j;
      if (k < ncr)
        c = c + df_make(v[j].x, v[j].y);
      else if (k < nch)
        r = r + df_make(v[j].x, v[j].y);
    }
  }
}

constexpr int kRedThreads = kReduceTargetsPerBlock * kRedLanes;
static_assert(kRedThreads == 256, "reduce block size");
static_assert(kRedLanes == 8, "sum_chunks strides by 8 lanes");

__global__ __launch_bounds__(kRedThreads) void k_reduce(const SysDev* __restrict__ sys, const int* __restrict__ sel,
                                                        const int2* __restrict__ sel_rng, int nsel,
                                                        const int2* __restrict__ items,
                                                        const float2* __restrict__ part,
                                                        const double* __restrict__ part64, int prec,
                                                        const double* __restrict__ q, const int* __restrict__ perm,
                                                        const double* __restrict__ r0,
                                                        double* __restrict__ phi_c, double* __restrict__ phi_r,
                                                        double* __restrict__ phi_t, double* __restrict__ epart,
                                                        double* __restrict__ energy, unsigned int* __restrict__ counter,
                                                        int* __restrict__ status, const OutDesc* __restrict__ out)
{
  __shared__ double red[2][kRedThreads / 32];
  __shared__ bool last;
  __shared__ int s_r;
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int n = S.n;
  // kRedLanes consecutive threads share a target: lane sub sums the chunks c = sub (mod
  // kRedLanes), then a fixed xor butterfly adds the lanes pairwise, so several
  // loads per target are in flight and the order does not depend on scheduling
  const int sub = threadIdx.x % kRedLanes;
  const int i = it.y * kReduceTargetsPerBlock + threadIdx.x / kRedLanes;
  // the target's input position, charge and the centre constant are loaded first (by every
  // lane of the target: one broadcast load), so their latency overlaps the partial sums
  long long o = 0;
  double qi = 0.0;
  const double rc = r0[it.x];
  if (i < n) {
    o = S.chg + perm[S.chg + i];  // partials are in sorted order
    qi = q[o];
  }
  // the caller's destinations (written by the host before the launch)
  const OutDesc od = out ? *out : OutDesc{nullptr, nullptr, 0, 0};
  // launch-local system r of this block (sel_rng ascending: the last r whose range starts at or
  // before this block), found by thread 0 before the wait
  int r_blk = 0, cnt_blk = 0;
  if (threadIdx.x == 0) {
    int lo = 0, hi = nsel - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sel_rng[mid].x <= (int)blockIdx.x)
        lo = mid;
      else
        hi = mid - 1;
    }
    r_blk = lo;
    cnt_blk = sel_rng[lo].y;
    s_r = lo;
  }
  // (launched as a programmatic dependent of the pair kernel: everything above reads data that
  // the pair sum does not write; the partials below wait for it)
  grid_dependency_wait();
  double et = 0.0, er = 0.0;
  const int nch = S.ncr + S.nck + S.ncs;
  if (prec == HSMA_FP64) {
    double pc = 0.0, pr = 0.0;
    if (i < n) {
      const double* b = part64 + S.part + i;
      for (int c = sub; c < S.ncr; c += kRedLanes) pc += b[(long long)c * n];
      for (int c = S.ncr + sub; c < nch; c += kRedLanes) pr += b[(long long)c * n];
    }
    for (int o = 1; o < kRedLanes; o <<= 1) {
      pc += __shfl_xor_sync(0xffffffffu, pc, o);
      pr += __shfl_xor_sync(0xffffffffu, pr, o);
    }
    if (i < n && sub == 0) {
      pr += rc;
      phi_c[o] = pc;
      phi_r[o] = pr;
      phi_t[o] = pc + pr;
      if (od.phi) od.phi[o] = od.what == 0 ? pc : (od.what == 1 ? pr : pc + pr);
      if (!isfinite(pc) || !isfinite(pr)) atomicOr(status, kStNonFinite);
      et = 0.5 * qi * (pc + pr);
      er = 0.5 * qi * pr;
    }
    for (int o = 16; o > 0; o >>= 1) {
      et += __shfl_xor_sync(0xffffffffu, et, o);
      er += __shfl_xor_sync(0xffffffffu, er, o);
    }
  } else {
    // the (hi, lo) partials, the centre constant and the energy terms in double-float
    // arithmetic on the FP32 pipes; FP64 only to convert (this GPU issues FP64 at a small
    // fraction of the FP32 rate), and the three conversions of a target spread over its lanes.  The
    // xor butterfly leaves the same sums in all kRedLanes lanes (df addition is commutative).
    df c = df_make(0.f, 0.f), r = df_make(0.f, 0.f);
    if (i < n) sum_chunks(part + S.part + i, n, sub, S.ncr, nch, c, r);
    for (int o = 1; o < kRedLanes; o <<= 1) {
      c = c + df_make(__shfl_xor_sync(0xffffffffu, c.hi, o), __shfl_xor_sync(0xffffffffu, c.lo, o));
      r = r + df_make(__shfl_xor_sync(0xffffffffu, r.hi, o), __shfl_xor_sync(0xffffffffu, r.lo, o));
    }
    r = r + df_from_double(rc);
    const df t = c + r;
    if (i < n && sub < 3) {
      double* dst = sub == 0 ? phi_c : (sub == 1 ? phi_r : phi_t);
      const double v = df_to_double(sub == 0 ? c : (sub == 1 ? r : t));
      dst[o] = v;
      if (od.phi && sub == od.what) od.phi[o] = v;
      if (sub == 0 && !(isfinite(c.hi) && isfinite(r.hi))) atomicOr(status, kStNonFinite);
    }
    const df hq = df_from_double(0.5 * qi);
    df ect = i < n && sub == 0 ? hq * t : df_make(0.f, 0.f);
    df ecr = i < n && sub == 0 ? hq * r : df_make(0.f, 0.f);
    for (int o = 16; o > 0; o >>= 1) {
      ect = ect + df_make(__shfl_xor_sync(0xffffffffu, ect.hi, o), __shfl_xor_sync(0xffffffffu, ect.lo, o));
      ecr = ecr + df_make(__shfl_xor_sync(0xffffffffu, ecr.hi, o), __shfl_xor_sync(0xffffffffu, ecr.lo, o));
    }
    if ((threadIdx.x & 31) == 0) {
      et = df_to_double(ect);
      er = df_to_double(ecr);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][warp] = et;
    red[1][warp] = er;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    for (int w = 0; w < kRedThreads / 32; ++w) {
      a += red[0][w];
      b += red[1][w];
    }
    epart[2 * blockIdx.x] = a;
    epart[2 * blockIdx.x + 1] = b;
    if (od.epart) {
      od.epart[2 * blockIdx.x] = a;
      od.epart[2 * blockIdx.x + 1] = b;
    }
    last = false;
    if (energy) {
      __threadfence();
      // whether this block is the last of its system's blocks to finish
      const unsigned prev = atomicAdd(&counter[r_blk], 1u);
      last = (prev == (unsigned)cnt_blk - 1u);
    }
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  // energies of system sel[r]: its blocks' partials in a fixed order (strided lanes, xor tree,
  // warps in order), so the result does not depend on which block finishes last
  const int r = s_r;
  const int2 rg = sel_rng[r];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < rg.y; k += kRedThreads) {
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
    for (int w = 0; w < kRedThreads / 32; ++w) {
      A += red[0][w];
      B += red[1][w];
    }
    energy[2 * sel[r]] = A;
    energy[2 * sel[r] + 1] = B;
    counter[r] = 0u;
  }
}

void launch_reduce(const SysDev* sys, const int* sel, const int2* sel_rng, int nsel, const int2* items, int nitems,
                   const float2* part, const double* part64, int prec, const double* q, const int* perm,
                   const double* r0, double* phi_c, double* phi_r, double* phi_t, double* epart, double* energy,
                   unsigned int* counter, int* status, const OutDesc* out, cudaStream_t st, bool pdl)
{
  if (nitems <= 0) return;
  launch_k(k_reduce, nitems, kRedThreads, 0, st, pdl, sys, sel, sel_rng, nsel, items, part, part64, prec, q, perm, r0,
           phi_c, phi_r, phi_t, epart, energy, counter, status, out);
}

}  // namespace hsma
