// Coulomb part of the pair sum for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all: code running inside a custom allocator or
// memory-pool callback (a nested allocation would re-enter the allocator), a plugin whose host
// application owns and accounts for all device memory, or a real-time loop whose memory budget
// is fixed up front.  For them this entry point computes
//   phi_i = k_over_eps1 * sum_{j != i} q_j / |x_i - x_j|
// with the tiled FP32 pair-sum kernel of the library (hi/lo split coordinates, one MUFU rsqrt
// per pair, compensated tile partials), but its scratch memory (the per-chunk partial sums and
// the completion counters) lives in a file-scope static __device__ array of fixed size, so the
// call allocates nothing.  That array exists on every GPU that loads the library until the
// process exits.
#include <cmath>
#include <mutex>

#include "fp32_pair.cuh"
#include "hsma_internal.cuh"

namespace hsma {
namespace {

constexpr int kNaThreads = 128;                 // CTA size
constexpr int kNaK = 2;                         // targets per thread
constexpr int kNaTB = kNaThreads * kNaK;        // targets per block
constexpr int kNaChunk = 1024;                  // sources per chunk
constexpr int kNaMaxN = HSMA_NOALLOC_MAX_N;     // largest n
constexpr int kNaMaxChunks = kNaMaxN / kNaChunk;
constexpr int kNaMaxTB = kNaMaxN / kNaTB;

// partial sums [chunk][target] as (hi, lo) and one completion counter per target block
struct __align__(256) NoAllocScratch {
  float2 part[(size_t)kNaMaxChunks * kNaMaxN];
  unsigned int done[kNaMaxTB];
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;


// One block per (target block, source chunk).  The last block of a target block to finish
// adds the chunk partials of its targets in chunk order (FP64) and writes phi.
__global__ __launch_bounds__(kNaThreads) void k_coulomb_noalloc(int n, const double* __restrict__ xyz,
                                                               const double* __restrict__ q, double kfac,
                                                               double* __restrict__ phi,
                                                               NoAllocScratch* __restrict__ scr)
{
  __shared__ float4 sh[kNaThreads], sl[kNaThreads];
  __shared__ bool last;
  const int nchunks = (n + kNaChunk - 1) / kNaChunk;
  const int tb = blockIdx.x / nchunks, c = blockIdx.x % nchunks;
  const int t0 = tb * kNaTB, tid = threadIdx.x;
  float th[kNaK][3], tl[kNaK][3];
  int ti[kNaK];
#pragma unroll
  for (int k = 0; k < kNaK; ++k) {
    const int i = t0 + k * kNaThreads + tid;
    const int ii = i < n ? i : t0;
    ti[k] = i;
    split_hilo(xyz[3 * (size_t)ii], th[k][0], tl[k][0]);
    split_hilo(xyz[3 * (size_t)ii + 1], th[k][1], tl[k][1]);
    split_hilo(xyz[3 * (size_t)ii + 2], th[k][2], tl[k][2]);
  }
  float H[kNaK], L[kNaK];
#pragma unroll
  for (int k = 0; k < kNaK; ++k) H[k] = L[k] = 0.f;
  const int s0 = c * kNaChunk, s1 = min(n, s0 + kNaChunk);
  for (int ts = s0; ts < s1; ts += kNaThreads) {
    const int cnt = min(kNaThreads, s1 - ts);
    if (tid < cnt) {
      const size_t j = (size_t)(ts + tid);
      float hx, hy, hz, lx, ly, lz;
      split_hilo(xyz[3 * j], hx, lx);
      split_hilo(xyz[3 * j + 1], hy, ly);
      split_hilo(xyz[3 * j + 2], hz, lz);
      sh[tid] = make_float4(hx, hy, hz, (float)(kfac * q[j]));
      sl[tid] = make_float4(lx, ly, lz, 0.f);
    }
    __syncthreads();
    float acc[kNaK];
#pragma unroll
    for (int k = 0; k < kNaK; ++k) acc[k] = 0.f;
    for (int s = 0; s < cnt; ++s) {
      const float4 h = sh[s], l = sl[s];
#pragma unroll
      for (int k = 0; k < kNaK; ++k) {
        const float dx = th[k][0] - h.x, dy = th[k][1] - h.y, dz = th[k][2] - h.z;
        const float ex = (tl[k][0] - l.x) + dx, ey = (tl[k][1] - l.y) + dy, ez = (tl[k][2] - l.z) + dz;
        float r2 = ex * ex;
        r2 = fmaf(ey, ey, r2);
        r2 = fmaf(ez, ez, r2);
        float inv = rsqrt_mufu(r2);
        inv = (ts + s == ti[k]) ? 0.f : inv;
        acc[k] = fmaf(h.w, inv, acc[k]);
      }
    }
#pragma unroll
    for (int k = 0; k < kNaK; ++k) {
      const float s = H[k] + acc[k];
      const float bp = s - H[k];
      L[k] += (H[k] - (s - bp)) + (acc[k] - bp);
      H[k] = s;
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < kNaK; ++k)
    if (ti[k] < n) scr->part[(size_t)c * kNaMaxN + ti[k]] = make_float2(H[k], L[k]);
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&scr->done[tb], 1u) == (unsigned)(nchunks - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int k = 0; k < kNaK; ++k) {
    if (ti[k] >= n) continue;
    double s = 0.0;
    for (int cc = 0; cc < nchunks; ++cc) {
      const float2 v = __ldcg(&scr->part[(size_t)cc * kNaMaxN + ti[k]]);
      s += (double)v.x + (double)v.y;
    }
    phi[ti[k]] = s;
  }
}

// Device address of the scratch array, looked up once per device (with that device current) and
// kept for the life of the process: it does not survive cudaDeviceReset, after which this entry
// point must not be called again in the same process.
std::mutex g_na_mutex;
void* g_na_addr[64] = {nullptr};

}  // namespace
}  // namespace hsma

extern "C" int hsma_coulomb_potential_noalloc(int64_t n, const double* xyz_dev, const double* q_dev,
                                              double k_over_eps1, double* phi_dev, void* stream)
{
  using namespace hsma;
  if (n < 0 || n > kNaMaxN) return HSMA_E_INVALID_ARG;
  if (n == 0) return HSMA_OK;
  if (!xyz_dev || !q_dev || !phi_dev || !std::isfinite(k_over_eps1)) return HSMA_E_INVALID_ARG;
  // an error left pending by earlier, unrelated work is the caller's: it is reported as such and
  // left in place (nothing is launched), so the checks below see only this call's own errors
  if (cudaPeekAtLastError() != cudaSuccess) return HSMA_E_CUDA;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return HSMA_E_CUDA;
  }
  void* addr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
      void* p = nullptr;
      if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return HSMA_E_CUDA;
      }
      g_na_addr[dev] = p;
    }
    addr = g_na_addr[dev];
  }
  NoAllocScratch* scr = static_cast<NoAllocScratch*>(addr);
  cudaStream_t st = (cudaStream_t)stream;
  const int ntb = (int)((n + kNaTB - 1) / kNaTB);
  const int nchunks = (int)((n + kNaChunk - 1) / kNaChunk);
  // the completion counters must start at zero; the partials are overwritten before use
  if (cudaMemsetAsync(scr->done, 0, sizeof(unsigned int) * ntb, st) != cudaSuccess) {
    cudaGetLastError();  // (this call's own error: none was pending on entry)
    return HSMA_E_CUDA;
  }
  k_coulomb_noalloc<<<ntb * nchunks, kNaThreads, 0, st>>>((int)n, xyz_dev, q_dev, k_over_eps1, phi_dev, scr);
  if (cudaGetLastError() != cudaSuccess) return HSMA_E_CUDA;  // the launch's own error
  return HSMA_OK;
}
