// Spatial order of the charges of every system, for the near/far split of the pair sum.
//
// Charges are sorted by the Morton index of their cell on a 16^3 grid over [-a, a]^3, and
// inside a cell by their key (the Morton index on a 2^key_lv grid: the cell's own index unless
// the far-field tree asks for a finer order) and then their input index, so the order (hence
// every summation order downstream) is deterministic.  Consecutive charges in this order are close in space: a warp's targets
// and a 32-source sub-tile each occupy a small box, and the pair kernel evaluates the pairs of
// well-separated boxes with plain FP32 coordinates, keeping the hi/lo-split form for near ones.
//   k_order_keys   cell key per charge and the cell histogram of its system (global integer
//                  atomics), the engine's own copy of device inputs read in place (InDesc),
//                  the check that the charge lies inside the cavity and, for the FP32
//                  path, the (hi, lo) split of its coordinates and charge (64-thread blocks: this
//                  is the FP64 arithmetic of the build's record chain, which this GPU issues at
//                  a low rate per SM, so it is spread over many SMs)
//   k_order_sort   sort_parts blocks per system, each owning a run of consecutive cells: every
//                  block scans the whole histogram (the system's last block to have read it
//                  zeroes it for the next build), reads all the system's keys (many loads in
//                  flight) and scatters those of its cells (atomic cursor in shared memory: any
//                  order inside a cell), then every slot finds its place in its cell by counting
//                  the cell's smaller input indices (the rank; cells hold a few charges), which
//                  gives perm (k_images, which reads perm on many SMs, writes its inverse)
// Two kernels and no memsets: the order is on the critical path of the overlapped step.
#include <algorithm>

#include "fp32_pair.cuh"
#include "hsma_internal.cuh"

namespace hsma {

__device__ __forceinline__ unsigned int spread3(unsigned int v)
{
  // interleave the 10 low bits of v with two zero bits each
  v &= 0x3FFu;
  v = (v | (v << 16)) & 0x030000FFu;
  v = (v | (v << 8)) & 0x0300F00Fu;
  v = (v | (v << 4)) & 0x030C30C3u;
  v = (v | (v << 2)) & 0x09249249u;
  return v;
}

// Morton index of the charge's cell on the 2^key_lv grid over [-a, a]^3
__device__ __forceinline__ int cell_key(const SysDev& S, double x, double y, double z)
{
  const int G = 1 << S.key_lv;
  const double s = 0.5 * G * S.inv_a;
  int ix = (int)floor((x + S.a) * s), iy = (int)floor((y + S.a) * s), iz = (int)floor((z + S.a) * s);
  ix = min(max(ix, 0), G - 1);
  iy = min(max(iy, 0), G - 1);
  iz = min(max(iz, 0), G - 1);
  return (int)(spread3((unsigned)ix) | (spread3((unsigned)iy) << 1) | (spread3((unsigned)iz) << 2));
}

constexpr int kKeyThreads = 64;
constexpr int kKeySplit = kOrderBlock / kKeyThreads;
__global__ __launch_bounds__(kKeyThreads) void k_order_keys(const SysDev* __restrict__ sys, const int2* __restrict__ items,
                                                            const InDesc* __restrict__ in,
                                                            double* __restrict__ xyz_own, double* __restrict__ q_own,
                                                            int* __restrict__ key, int* __restrict__ hist,
                                                            float4* __restrict__ xs, int* __restrict__ status,
                                                            unsigned int* __restrict__ ctr_reset, int nreset)
{
  if (blockIdx.x == 0 && (int)threadIdx.x < nreset) ctr_reset[threadIdx.x] = 0u;
  const int2 it = items[blockIdx.x / kKeySplit];
  const SysDev& S = sys[it.x];
  const int i = it.y * kOrderBlock + (blockIdx.x % kKeySplit) * kKeyThreads + threadIdx.x;
  if (i >= S.n) return;
  const long long g = S.chg + i;
  const InDesc d = *in;
  const double x = d.xyz[3 * g], y = d.xyz[3 * g + 1], z = d.xyz[3 * g + 2], qg = d.q[g];
  if (d.copy) {
    // the engine's own copy of the inputs, which the later kernels of the pass read
    xyz_own[3 * g] = x;
    xyz_own[3 * g + 1] = y;
    xyz_own[3 * g + 2] = z;
    q_own[g] = qg;
  }
  const int k = cell_key(S, x, y, z);
  key[g] = k;
  atomicAdd(&hist[(size_t)it.x * kOrderCells + (k >> (3 * (S.key_lv - kOrderLevels)))], 1);
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
  if (!(r2 < S.a * S.a) || !isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(qg)) atomicOr(status, kStOutside);
  if (xs) {
    const float2 sx = split_pair(x), sy = split_pair(y), sz = split_pair(z), sq = split_pair(qg);
    xs[2 * g] = make_float4(sx.x, sy.x, sz.x, sq.x);
    xs[2 * g + 1] = make_float4(sx.y, sy.y, sz.y, sq.y);
  }
}

// Blocks of a system: part it.y of S.sort_parts takes cells [k0, k1), k1 - k0 = kOrderCells /
// sort_parts, i.e. sorted positions [P0, P1).  s_cell holds the first sorted position of every
// cell (exclusive scan of the histogram), then (after the scatter) the end of each of the
// block's cells.  The block's scattered slots (input index and cell) live in shared memory when
// they are at most smem_n (the launch's dynamic shared memory, sized by the engine), else in the
// scratch buffer scr (2 ints per charge of the system: input indices, then cells).  done[s]
// counts the system's blocks that have read the histogram; the last one zeroes both.
constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortBatch = 8;  // keys in flight per thread
static_assert(kOrderCells % kSortThreads == 0, "cells split evenly over the sort block");

__global__ __launch_bounds__(kSortThreads) void k_order_sort(const SysDev* __restrict__ sys,
                                                             const int2* __restrict__ items,
                                                             const int* __restrict__ key, int* __restrict__ hist,
                                                             int* __restrict__ done, int* __restrict__ scr,
                                                             int* __restrict__ perm, int smem_n)
{
  __shared__ int s_cell[kOrderCells];
  __shared__ int s_wsum[kSortWarps];
  __shared__ int s_last;
  extern __shared__ int s_slot[];
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int n = S.n, parts = S.sort_parts;
  const int ksh = 3 * (S.key_lv - kOrderLevels);  // key -> cell
  const long long c0 = S.chg;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // k_images, a programmatic dependent of this kernel, is dispatched right away and waits for
  // this grid (a programmatic launch of this kernel after k_order_keys put both blocks on one
  // SM beside a moment block: 3 us slower)
  allow_dependents();
  int* h = hist + (size_t)it.x * kOrderCells;

  // exclusive scan: thread t owns cells [t per, (t + 1) per)
  constexpr int per = kOrderCells / kSortThreads;
  int cnt[per];
  int sum = 0;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    cnt[j] = h[tid * per + j];
    sum += cnt[j];
  }
  if (parts == 1) {
#pragma unroll
    for (int j = 0; j < per; ++j) h[tid * per + j] = 0;  // (read by this block alone)
  }
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) s_wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = lane < kSortWarps ? s_wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += v;
    }
    if (lane < kSortWarps) s_wsum[lane] = w;
  }
  if (parts > 1 && tid == 0) s_last = atomicAdd(&done[it.x], 1) == parts - 1;
  __syncthreads();
  int run = incl - sum + (warp > 0 ? s_wsum[warp - 1] : 0);
#pragma unroll
  for (int j = 0; j < per; ++j) {
    s_cell[tid * per + j] = run;
    run += cnt[j];
  }
  if (parts > 1 && s_last) {
    // every block of the system has read the histogram (each counted itself after its scan)
#pragma unroll
    for (int j = 0; j < per; ++j) h[tid * per + j] = 0;
    if (tid == 0) done[it.x] = 0;
  }
  __syncthreads();

  const int k0 = it.y * (kOrderCells / parts), k1 = k0 + kOrderCells / parts;
  const int P0 = s_cell[k0], P1 = k1 < kOrderCells ? s_cell[k1] : n;
  const int m = P1 - P0;
  int* slot = m <= smem_n ? s_slot : scr + 2 * c0 + P0;
  int* skey = m <= smem_n ? s_slot + smem_n : scr + 2 * c0 + n + P0;
  __syncthreads();  // P0 is read before the cursors move

  // scatter the keys of the block's cells
  for (int i0 = 0; i0 < n; i0 += kSortBatch * kSortThreads) {
    int kk[kSortBatch];
#pragma unroll
    for (int j = 0; j < kSortBatch; ++j) {
      const int i = i0 + j * kSortThreads + tid;
      kk[j] = i < n ? key[c0 + i] : -1;
    }
#pragma unroll
    for (int j = 0; j < kSortBatch; ++j) {
      const int cell = kk[j] >> ksh;  // (-1 stays -1)
      if (cell >= k0 && cell < k1) {
        const int p = atomicAdd(&s_cell[cell], 1) - P0;
        slot[p] = i0 + j * kSortThreads + tid;
        skey[p] = kk[j];
      }
    }
  }
  __syncthreads();

  // slot a of cell k (which spans [end of cell k - 1, end of cell k), the first from P0) goes to
  // the cell's start plus the number of the cell's charges before it: the input indices below
  // its own or, with a finer key, the (key, input index) pairs below its own
  for (int a = tid; a < m; a += kSortThreads) {
    const int v = slot[a], kf = skey[a], k = kf >> ksh;
    const int b0 = (k > k0 ? s_cell[k - 1] : P0) - P0, e = s_cell[k] - P0;
    int p = b0;
    if (ksh == 0) {
      for (int b = b0; b < e; ++b) p += slot[b] < v;
    } else {
      for (int b = b0; b < e; ++b) {
        const int kb = skey[b];
        p += kb < kf || (kb == kf && slot[b] < v);
      }
    }
    perm[c0 + P0 + p] = v;
  }
}

void init_order_kernels()
{
  cudaFuncSetAttribute(k_order_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * sizeof(int) * kOrderSmemMaxN);
}

int order_sort_parts(int64_t n)
{
  int parts = 1;
  while (parts < kSortMaxParts && (int64_t)parts * kSortPartCharges < n) parts *= 2;
  return parts;
}

int order_smem_charges(int64_t max_n)
{
  int64_t c = std::max<int64_t>(4096, (max_n + 1023) / 1024 * 1024);
  return (int)std::min<int64_t>(c, kOrderSmemMaxN);
}

void launch_order(const SysDev* sys, int nsys, const int2* items, int nitems, const int2* sitems, int nsitems,
                  const InDesc* in, double* xyz_own, double* q_own, int* key, int* hist, int* scr, int* perm,
                  float4* xs, int* status, unsigned int* ctr_reset, int nreset, int smem_n, cudaStream_t st)
{
  if (nitems <= 0 || nsys <= 0 || nsitems <= 0) return;
  launch_k(k_order_keys, nitems * kKeySplit, kKeyThreads, 0, st, false, sys, items, in, xyz_own, q_own, key, hist,
           xs, status, ctr_reset, nreset);
  launch_k(k_order_sort, nsitems, kSortThreads, 2 * sizeof(int) * (size_t)smem_n, st, false, sys, sitems,
           (const int*)key, hist, hist + (size_t)nsys * kOrderCells, scr, perm, smem_n);
}

}  // namespace hsma
