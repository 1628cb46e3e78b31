// Treecode far field of the real-charge and Kelvin-image pair sums of one large cavity (FP32
// path): the multipole acceleration the paper applies to the pair sum of eq. phirffinall for
// N up to 1e6 (Sec. 4.2, Algorithm 1 step 5), done here as a GPU treecode over the spatial order
// of the records.  Kernels in k_tree.cu.
#pragma once

#include <cuda_runtime.h>

#include "hsma_internal.cuh"

namespace hsma {

// Octree levels 0..L over the cube [-a, a]^3 of the cavity: node (l, c) is cell c (Morton
// index) of the 2^l per axis grid; its records are the sorted positions whose key has the
// prefix c (a contiguous range, because records are in Morton order of a grid at least as fine,
// 2^key_lv per axis).  Dense per-level arrays: node (l, c) sits at tree_node_index(l, c).
constexpr int kTreeTop = 2;       // traversal roots: the 64 cells of level 2
constexpr int kTreeRootSplit = 8; // work items per (group, tree): the roots in this many runs
constexpr int kTreeMaxLevel = 7;  // finest node level supported
constexpr int kFarOrder = 24;     // order of the origin-centred expansion of the far images
constexpr float kFarImageRel = 2.0f;  // Kelvin images beyond this multiple of a: far images
constexpr int kTreeEvalWarps = 4;     // warps (persistent target-group workers) per k_tree_eval block
constexpr int kTreeEvalMinBlocks = 7; // resident k_tree_eval blocks per SM the kernel is built for
constexpr int kTreeStack = 128;       // traversal stack entries per warp
constexpr int kFarBlocks = 512;       // blocks of k_tree_far

__host__ __device__ constexpr long long tree_node_index(int l, long long c) { return ((1LL << (3 * l)) - 1) / 7 + c; }
__host__ __device__ constexpr long long tree_node_count(int L) { return ((1LL << (3 * (L + 1))) - 1) / 7; }
__host__ __device__ constexpr int tree_nm(int P) { return (P + 1) * (P + 2) / 2; }  // complex moments n <= P, 0 <= m <= n

// Everything the tree kernels read and write (device pointers into the engine's workspace;
// one system).
struct TreeView {
  const SysDev* sys;         // the system (index 0)
  const int* key;            // fine Morton key per input charge (k_order_keys)
  const int* perm;           // sorted position -> input index
  const float4* hi;          // records (x_hi, y_hi, z_hi, Q): real at [src, src + n), Kelvin after
  const float4* lo;          // (x_lo, y_lo, z_lo, .)
  int2* node;                // [nodes]: record range [begin, end) of every node
  float4* geo;               // [2][nodes]: centre and radius of the real / Kelvin sources (radius < 0: none)
  float4* box;               // [2][nodes][2]: bounding box (min, max) of the same
  float2* mom;               // [2][nodes][nm]: multipole moments about the centre, in units of the radius
  float2* farp;              // [kFarBlocks][tree_nm(kFarOrder)]: block partials of the far-image expansion
  float2* farL;              // [tree_nm(kFarOrder)]: the far-image expansion
  unsigned int* ctr;         // [0]: completion counter of k_tree_far, [1]: k_tree_eval's work counter
  int L;                     // finest node level
  int key_lv;                // levels of the record order's key (>= L)
  int P;                     // multipole order
  int cmin;                  // smallest node that is evaluated through its moments
  float theta;               // opening criterion: a node is far from a target group when
                             // radius of node <= theta * (distance of each target from its centre)
  float log_eps;             // log(0.1 theta^(P+1)): the truncation bound of a node's series
  float rfar2;               // (kFarImageRel a)^2
  float inv_a;
};

int tree_levels(long long n);
bool tree_order_supported(int P);
void launch_tree_build(const TreeView& t, int n, cudaStream_t st);
void launch_tree_eval(const TreeView& t, int n, float2* part, cudaStream_t st);

}  // namespace hsma
