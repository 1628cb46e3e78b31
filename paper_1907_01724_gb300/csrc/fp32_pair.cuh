// Device helpers of the FP32 pair sums (pair, field, move and allocation-free kernels): the MUFU
// reciprocal square root, cp.async staging, and the (hi, lo) FP32 split of an FP64 value.
#pragma once
#include <cuda_runtime.h>

#include "df64.cuh"

namespace hsma {

// 1/sqrt(x) by one MUFU instruction (rsqrt.approx, ~2^-22.9 relative; flushes subnormals).
__device__ __forceinline__ float rsqrt_mufu(float x)
{
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 16-byte asynchronous global -> shared copy (both addresses 16-byte aligned), its commit group
// and the wait for all but the N most recent groups.
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

// x = hi + lo to ~2^-48 relative: hi = fl32(x), lo = fl32(x - hi) (split_double, df64.cuh).
__device__ __forceinline__ void split_hilo(double x, float& hi, float& lo) { split_double(x, hi, lo); }
__device__ __forceinline__ float2 split_pair(double x)
{
  float2 r;
  split_hilo(x, r.x, r.y);
  return r;
}

// 1/|a - b| of two hi/lo-split points: with dh the FP32 difference of the high parts (exact for
// nearby points) and dl that of the low parts, dh + dl is the coordinate difference to FP32
// relative accuracy at any distance.
__device__ __forceinline__ float inv_hilo(float ax, float ay, float az, float alx, float aly, float alz, float bx,
                                          float by, float bz, float blx, float bly, float blz)
{
  const float dx = ax - bx, dy = ay - by, dz = az - bz;
  const float ex = (alx - blx) + dx, ey = (aly - bly) + dy, ez = (alz - blz) + dz;
  float r2 = ex * ex;
  r2 = fmaf(ey, ey, r2);
  r2 = fmaf(ez, ez, r2);
  return rsqrt_mufu(r2);
}

}  // namespace hsma
