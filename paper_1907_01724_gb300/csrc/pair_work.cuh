// Work lists of the persistent pair and field kernels and how a CTA takes its next item.
#pragma once
#include <cuda_runtime.h>

namespace hsma {

// A list of pair work items.  Items [0, first) are the first items of workers 0 .. first - 1 of
// the launch that has the list as w1 (a worker is a CTA, or a warp of the FP32 pair kernel; no
// atomic: a grid-wide first fetch from one counter serialises thousands of atomics); the rest are
// pulled through an atomic counter (zero before the first launch that uses it) as first +
// counter.  counter == nullptr: no list.
struct PairWork {
  const int4* items;
  int nitems;
  unsigned int* counter;
  int first;
};
// An item from the counter of w, or -1 when none is left (a plain read first: a list that is
// already exhausted costs no atomic, so CTAs that find no work do not queue on the counter).
__device__ __forceinline__ int pull_pair_item(const PairWork& w)
{
  if (!w.counter || w.first >= w.nitems) return -1;
  if (w.first + (int)__ldcg(w.counter) >= w.nitems) return -1;
  const int v = w.first + (int)atomicAdd(w.counter, 1u);
  return v < w.nitems ? v : -1;
}

// Next work item of a persistent CTA (thread 0): items of w1 first (the CTA's own item of the
// static round on its first fetch, then the counter), then, when w1 is exhausted, items of w2
// (if any).  list = 0 or 1 names the list of the item, 2 means no work left.
__device__ __forceinline__ void next_pair_item(const PairWork& w1, const PairWork& w2, int list,
                                               bool first_fetch, int& s_item, int& s_list)
{
  int v = 0;
  if (list == 0) {
    v = first_fetch && (int)blockIdx.x < w1.first ? (int)blockIdx.x : pull_pair_item(w1);
    if (v < 0) list = 1;
  }
  if (list == 1) {
    v = pull_pair_item(w2);
    if (v < 0) list = 2;
  }
  s_item = v;
  s_list = list;
}

}  // namespace hsma
