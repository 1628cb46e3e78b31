// Reduction of the pair-sum partials to potentials and energies (Algorithm 1 step 5 and the
// energy of Sec. 4, Fu & Gan, arXiv:1907.01724): one compensated FP32 (hi, lo) partial per
// (source chunk, target) on the FP32 path, one FP64 value on the FP64 path, written by
// k_pairs_f32 / k_pairs_f64 in the spatial order of k_order.cu; the results go to input order.
#include <math.h>

#include "df64.cuh"
#include "hsma_internal.cuh"

namespace hsma {

// phi_coul = sum of real-chunk partials, phi_rf = Kelvin + surface partials + centre constant,
// energies E_total = 1/2 sum q (phi_coul + phi_rf), E_RF = 1/2 sum q phi_rf.  Fixed-order
// block reductions; the last block of a system to finish (counter[r] per launch-local system
// r, reset by that block) sums the system's block partials in a fixed order.
constexpr int kRedLanes = 4;
// Sum of the (hi, lo) partials of chunks k = k0, k0 + kRedLanes, ... < k1 in ascending order
// into acc: kRedBatch chunks' loads are issued ahead of their additions, so a target's
// partials cost a few L2 round trips instead of one per chunk (slots past k1 add zero).
constexpr int kRedBatch = 8;
__device__ __forceinline__ void sum_range(const float2* __restrict__ b, long long n, int k0, int k1, df& acc)
{
  for (; k0 < k1; k0 += kRedBatch * kRedLanes) {
    float2 v[kRedBatch];
#pragma unroll
    for (int j = 0; j < kRedBatch; ++j) {
      const int k = k0 + kRedLanes * j;
      v[j] = k < k1 ? b[(long long)k * n] : make_float2(0.f, 0.f);
    }
#pragma unroll
    for (int j = 0; j < kRedBatch; ++j) acc = acc + df_make(v[j].x, v[j].y);
  }
}
// This lane's chunks (k = sub mod kRedLanes): the real chunks (k < ncr) into c, the others into
// r.  (Four lanes per target: the lanes' shared work per target -- the butterfly, the
// conversions and the energy terms -- is paid by half as many lanes as with eight.)
__device__ __forceinline__ void sum_chunks(const float2* __restrict__ b, long long n, int sub, int ncr, int nch,
                                           df& c, df& r)
{
  sum_range(b, n, sub, ncr, c);
  const int k2 = ncr + ((sub - ncr) % kRedLanes + kRedLanes) % kRedLanes;  // first k >= ncr, k = sub mod lanes
  sum_range(b, n, k2, nch, r);
}

constexpr int kRedThreads = kReduceTargetsPerBlock * kRedLanes;
static_assert(kRedThreads == 128, "reduce block size");
static_assert(kRedLanes >= 3, "lanes 0, 1, 2 of a target write phi_c, phi_r, phi_t");

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
  __shared__ float2 red2[2][kRedThreads / 32];
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
  const OutDesc od = out ? *out : OutDesc{nullptr, nullptr, nullptr, 0, 0};
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
  if (od.status && blockIdx.x == 0 && threadIdx.x == 0) {
    // the flags of the pass's earlier kernels (all complete here), for the caller's host copy
    const int st = __ldcg(status);
    for (int b = 0; b < kStBits; ++b)
      if (st & (1 << b)) od.status[b] = 1;
  }
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
      if (!isfinite(pc) || !isfinite(pr)) {
        atomicOr(status, kStNonFinite);
        if (od.status) od.status[1] = 1;
      }
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
      if (sub == 0 && !(isfinite(c.hi) && isfinite(r.hi))) {
        atomicOr(status, kStNonFinite);
        if (od.status) od.status[1] = 1;
      }
    }
    // q/2 split exactly (halving a split is exact away from underflow)
    const df q1 = df_from_double(qi), hq = df_make(0.5f * q1.hi, 0.5f * q1.lo);
    df ect = i < n && sub == 0 ? hq * t : df_make(0.f, 0.f);
    df ecr = i < n && sub == 0 ? hq * r : df_make(0.f, 0.f);
    for (int o = 16; o > 0; o >>= 1) {
      ect = ect + df_make(__shfl_xor_sync(0xffffffffu, ect.hi, o), __shfl_xor_sync(0xffffffffu, ect.lo, o));
      ecr = ecr + df_make(__shfl_xor_sync(0xffffffffu, ecr.hi, o), __shfl_xor_sync(0xffffffffu, ecr.lo, o));
    }
    if ((threadIdx.x & 31) == 0) {
      red2[0][threadIdx.x >> 5] = make_float2(ect.hi, ect.lo);
      red2[1][threadIdx.x >> 5] = make_float2(ecr.hi, ecr.lo);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0 && prec == HSMA_FP64) {
    red[0][warp] = et;
    red[1][warp] = er;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, b = 0.0;
    if (prec == HSMA_FP64) {
      for (int w = 0; w < kRedThreads / 32; ++w) {
        a += red[0][w];
        b += red[1][w];
      }
    } else {
      // the warps' double-float sums in order, one conversion per block
      df A = df_make(0.f, 0.f), B = df_make(0.f, 0.f);
      for (int w = 0; w < kRedThreads / 32; ++w) {
        A = A + df_make(red2[0][w].x, red2[0][w].y);
        B = B + df_make(red2[1][w].x, red2[1][w].y);
      }
      a = df_to_double(A);
      b = df_to_double(B);
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
  if (prec == HSMA_FP64) {
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
    return;
  }
  // FP32 path: the block partials in double-float (the FP64 additions of one block would queue
  // on its SM's FP64 unit at the end of the pass)
  df a = df_make(0.f, 0.f), b = df_make(0.f, 0.f);
  for (int k = threadIdx.x; k < rg.y; k += kRedThreads) {
    a = a + df_from_double(__ldcg(&epart[2 * (rg.x + k)]));
    b = b + df_from_double(__ldcg(&epart[2 * (rg.x + k) + 1]));
  }
  for (int o = 16; o > 0; o >>= 1) {
    a = a + df_make(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
    b = b + df_make(__shfl_xor_sync(0xffffffffu, b.hi, o), __shfl_xor_sync(0xffffffffu, b.lo, o));
  }
  __syncthreads();
  if (lane == 0) {
    red2[0][warp] = make_float2(a.hi, a.lo);
    red2[1][warp] = make_float2(b.hi, b.lo);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    df A = df_make(0.f, 0.f), B = df_make(0.f, 0.f);
    for (int w = 0; w < kRedThreads / 32; ++w) {
      A = A + df_make(red2[0][w].x, red2[0][w].y);
      B = B + df_make(red2[1][w].x, red2[1][w].y);
    }
    energy[2 * sel[r]] = df_to_double(A);
    energy[2 * sel[r] + 1] = df_to_double(B);
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
