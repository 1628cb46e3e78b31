// Direct tiled Coulomb sum of HSMA (Algorithm 1 step 5, eq. phirffinall of Fu & Gan,
// arXiv:1907.01724).
//
// Sources of one cavity: n real charges (excluding the target itself), n trapezoid-modified
// Kelvin images, and M surface points each carrying a monopole and a dipole (the 3M discrete
// images of eq. phicorrfinall).  Work is split into items (system, target block, source
// chunk); persistent workers (CTAs on the FP64 path, warps on the FP32 path) pull items from an
// atomic counter (longest items first) and write one compensated partial per (chunk, target),
// which k_reduce (k_reduce.cu) sums in a fixed order (FP64, or double-float on the FP32 path),
// so results do not depend on scheduling.  Records and partials are in the spatial order of
// k_order.cu; k_reduce maps them back to input order.  On the FP32 path the real and Kelvin
// items cover each unordered pair of blocks once and fill both blocks' slots (k_pairs_f32.cuh).
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
#include "fp32_pair.cuh"
#include "hsma_internal.cuh"

namespace hsma {

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

// Tile configurations: kernel variants (CTA threads, targets per thread), each with 4, 2, 1 or 8
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
static const int kItemsPerSlot[] = {4, 2, 1, 8};
constexpr int kItemChoices = (int)(sizeof(kItemsPerSlot) / sizeof(kItemsPerSlot[0]));

int pair_config_count() { return kPairKernels * kItemChoices; }
int pair_workers_per_cta(int cfg) { return kPairKernel[cfg % kPairKernels][0] / 32; }
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
  case i: cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pairs_f32<nt, k>, nt, pair_dyn_smem(nt)); break;
    HSMA_PAIR_CONFIGS(HSMA_CFG_OCC)
#undef HSMA_CFG_OCC
    default: break;
  }
  return b;
}

// registers a CTA of the configuration holds (the per-thread count in allocation units of 8)
int pairs_f32_block_regs(int cfg)
{
  cudaFuncAttributes a{};
  int nt = 0;
  switch (pair_kernel_of(cfg)) {
#define HSMA_CFG_REGS(i, t, k) \
  case i: cudaFuncGetAttributes(&a, k_pairs_f32<t, k>); nt = t; break;
    HSMA_PAIR_CONFIGS(HSMA_CFG_REGS)
#undef HSMA_CFG_REGS
    default: break;
  }
  return (a.numRegs + 7) / 8 * 8 * nt;
}

void launch_pairs_f32(int cfg, int grid, const SysDev* sys, PairWork w1, PairWork w2, const float4* src_hi,
                      const float4* src_lo, const float4* surf_a, const float4* surf_b, const float4* boxes,
                      float2* part, cudaStream_t st, bool pdl)
{
  switch (pair_kernel_of(cfg)) {
#define HSMA_CFG_LAUNCH(i, nt, k)                                                                          \
  case i:                                                                                                  \
    launch_k(k_pairs_f32<nt, k>, grid, nt, pair_dyn_smem(nt), st, pdl, sys, w1, w2, src_hi, src_lo, surf_a, surf_b, \
             boxes, part);                                                                                 \
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
                      const dbl4* surf64_a, const double* surf64_b, double* part64, cudaStream_t st, bool pdl)
{
  launch_k(k_pairs_f64, grid, kF64Threads, 0, st, pdl, sys, w1, w2, src64, surf64_a, surf64_b, part64);
}

}  // namespace hsma
