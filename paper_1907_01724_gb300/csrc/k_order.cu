// Spatial order of the charges of every system, for the near/far split of the pair sum.
//
// Charges are sorted by the Morton index of their cell on a 16^3 grid over [-a, a]^3, and
// inside a cell by their input index, so the order (hence every summation order downstream)
// is deterministic.  Consecutive charges in this order are close in space: a warp's targets
// and a 32-source sub-tile each occupy a small box, and the pair kernel evaluates the pairs of
// well-separated boxes with plain FP32 coordinates, keeping the hi/lo-split form for near ones.
//   k_order_cells    cell key per charge, histogram per system (integer atomics: exact)
//   k_order_scan     exclusive scan of each system's histogram (one block per system)
//   k_order_scatter  charge -> slot of its cell (atomic cursor: any order inside a cell)
//   k_order_sort     sort every cell's slots by input index (insertion sort; cells are small)
//                    and write the inverse permutation
#include "hsma_internal.cuh"

namespace hsma {

__device__ __forceinline__ unsigned int spread3(unsigned int v)
{
  // interleave the 4 low bits of v with two zero bits each
  v &= 0xFu;
  v = (v | (v << 4)) & 0x0C3u;
  v = (v | (v << 2)) & 0x249u;
  return v;
}

__device__ __forceinline__ int cell_key(const SysDev& S, double x, double y, double z)
{
  const double s = 0.5 * kOrderGrid * S.inv_a;
  int ix = (int)floor((x + S.a) * s), iy = (int)floor((y + S.a) * s), iz = (int)floor((z + S.a) * s);
  ix = min(max(ix, 0), kOrderGrid - 1);
  iy = min(max(iy, 0), kOrderGrid - 1);
  iz = min(max(iz, 0), kOrderGrid - 1);
  return (int)(spread3((unsigned)ix) | (spread3((unsigned)iy) << 1) | (spread3((unsigned)iz) << 2));
}

__global__ __launch_bounds__(kOrderBlock) void k_order_cells(const SysDev* __restrict__ sys, const int2* __restrict__ items,
                                                     const double* __restrict__ xyz, int* __restrict__ key,
                                                     int* __restrict__ hist)
{
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int i = it.y * kOrderBlock + threadIdx.x;
  if (i >= S.n) return;
  const long long g = S.chg + i;
  const int k = cell_key(S, xyz[3 * g], xyz[3 * g + 1], xyz[3 * g + 2]);
  key[g] = k;
  atomicAdd(&hist[(size_t)it.x * kOrderCells + k], 1);
}

// exclusive scan of kOrderCells counts with 1024 threads (4 cells per thread)
__global__ __launch_bounds__(1024) void k_order_scan(int nsys, const int* __restrict__ hist, int* __restrict__ offs,
                                                     int* __restrict__ cursor)
{
  __shared__ int warp_sums[32];
  const int s = blockIdx.x;
  if (s >= nsys) return;
  const int* h = hist + (size_t)s * kOrderCells;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  constexpr int per = kOrderCells / 1024;
  int local[per];
  int sum = 0;
#pragma unroll
  for (int j = 0; j < per; ++j) {
    local[j] = h[t * per + j];
    sum += local[j];
  }
  int incl = sum;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) warp_sums[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int w = warp_sums[lane];
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += v;
    }
    warp_sums[lane] = w;
  }
  __syncthreads();
  int run = incl - sum + (warp > 0 ? warp_sums[warp - 1] : 0);
#pragma unroll
  for (int j = 0; j < per; ++j) {
    offs[(size_t)s * kOrderCells + t * per + j] = run;
    cursor[(size_t)s * kOrderCells + t * per + j] = run;
    run += local[j];
  }
}

__global__ __launch_bounds__(kOrderBlock) void k_order_scatter(const SysDev* __restrict__ sys, const int2* __restrict__ items,
                                                       const int* __restrict__ key, int* __restrict__ cursor,
                                                       int* __restrict__ perm)
{
  const int2 it = items[blockIdx.x];
  const SysDev& S = sys[it.x];
  const int i = it.y * kOrderBlock + threadIdx.x;
  if (i >= S.n) return;
  const int pos = atomicAdd(&cursor[(size_t)it.x * kOrderCells + key[S.chg + i]], 1);
  perm[S.chg + pos] = i;
}

// one thread per cell: insertion sort of the cell's slots by input index, then the inverse map
__global__ __launch_bounds__(256) void k_order_sort(const SysDev* __restrict__ sys, int nsys,
                                                    const int* __restrict__ hist, const int* __restrict__ offs,
                                                    int* __restrict__ perm, int* __restrict__ iperm)
{
  const long long gid = (long long)blockIdx.x * 256 + threadIdx.x;
  const int s = (int)(gid / kOrderCells);
  const int c = (int)(gid % kOrderCells);
  if (s >= nsys) return;
  const SysDev& S = sys[s];
  const int cnt = hist[(size_t)s * kOrderCells + c];
  if (cnt == 0) return;
  int* seg = perm + S.chg + offs[(size_t)s * kOrderCells + c];
  for (int a = 1; a < cnt; ++a) {
    const int v = seg[a];
    int b = a - 1;
    while (b >= 0 && seg[b] > v) {
      seg[b + 1] = seg[b];
      --b;
    }
    seg[b + 1] = v;
  }
  const int base = offs[(size_t)s * kOrderCells + c];
  for (int a = 0; a < cnt; ++a) iperm[S.chg + seg[a]] = base + a;
}

void launch_order(const SysDev* sys, int nsys, const int2* items, int nitems, const double* xyz, int* key, int* hist,
                  int* offs, int* cursor, int* perm, int* iperm, cudaStream_t st)
{
  if (nitems <= 0 || nsys <= 0) return;
  cudaMemsetAsync(hist, 0, sizeof(int) * (size_t)nsys * kOrderCells, st);
  k_order_cells<<<nitems, kOrderBlock, 0, st>>>(sys, items, xyz, key, hist);
  k_order_scan<<<nsys, 1024, 0, st>>>(nsys, hist, offs, cursor);
  k_order_scatter<<<nitems, kOrderBlock, 0, st>>>(sys, items, key, cursor, perm);
  const long long cells = (long long)nsys * kOrderCells;
  k_order_sort<<<(int)((cells + 255) / 256), 256, 0, st>>>(sys, nsys, hist, offs, perm, iperm);
}

}  // namespace hsma
