// Internal declarations shared by the CUDA translation units of the HSMA library.
// Layout, per-system descriptors and kernel launchers.  Nothing here is part of the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/hsma.h"

#include "pair_work.cuh"

namespace hsma {

constexpr double kPi = 3.14159265358979323846264338327950288;

// 32-byte FP64 record (position + strength) for the FP64 path.
struct __align__(32) dbl4 {
  double x, y, z, w;
};
__host__ __device__ __forceinline__ dbl4 make_dbl4(double x, double y, double z, double w)
{
  dbl4 r;
  r.x = x;
  r.y = y;
  r.z = z;
  r.w = w;
  return r;
}

// Status bits written by kernels (the host maps them to HSMA_E_* codes).  No kernel of the
// library waits on another CTA or on the host, so none has a timeout status.
enum : int {
  kStOutside = 1,    // a charge at |x| >= a or with a non-finite coordinate
  kStNonFinite = 2,  // a non-finite potential
  kStBadMove = 8,    // delta-energy move target outside the cavity
};

// Charges closer to the centre than this fraction of a use the r_K -> infinity limit of
// their Kelvin image (a constant potential); the limit differs from the image term by a
// relative O(r |x| / a^2) <= 1e-12.
constexpr double kCentreRel = 1e-12;

// Programmatic dependent launch: a kernel launched with launch_pdl may start while its
// predecessor in the stream is finishing; it calls grid_dependency_wait() before it reads
// anything the predecessor writes (a no-op when launched normally).  A predecessor lets its
// dependent launch early with allow_dependents().
__device__ __forceinline__ void grid_dependency_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void allow_dependents() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Launch priority (a stream-priority value, 0 = the default, lower = more urgent) that the
// launchers below give their kernels; the engine sets it around each launcher call, so that in
// the overlapped step the work that gates the pair sum is dispatched before the pair sum of the
// real and Kelvin records, which runs beside it.  Graphs are instantiated to honour it.
int& launch_priority();
struct PriorityScope {
  int saved;
  explicit PriorityScope(int p) : saved(launch_priority()) { launch_priority() = p; }
  ~PriorityScope() { launch_priority() = saved; }
};

// Kernel launch with the current launch priority and, when pdl is set, programmatic dependent
// launch.
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st, bool pdl,
                     Args... args)
{
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[2];
  unsigned na = 0;
  if (pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (launch_priority() != 0) {
    attr[na].id = cudaLaunchAttributePriority;
    attr[na].val.priority = launch_priority();
    ++na;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                       Args... args)
{
  launch_k(kern, grid, block, smem, st, true, args...);
}

// Per-system descriptor, resident on the device.  The host fills the inputs and the layout
// offsets; k_setup fills the derived scalars (Sec. 2.3/2.4).
struct SysDev {
  // inputs (Sec. 2.1 and the numerical parameters)
  double a, eps1, eps2, kappa, tau, dy_rel, coulk;
  // derived on the device by k_setup
  double eps, mu, Rtau, dy, gam, sig, dbar, kc;  // kc = coulk / eps1
  double inv_a, kc_a, Rt_a, inv_Rt;              // 1/a, kc/a, R_tau/a, 1/R_tau
  int p, P, M, F1, F2;
  int n;              // charges
  int prec;           // HSMA_FP32 / HSMA_FP64
  int sort_parts;     // blocks of k_order_sort for this system (a power of two; each sorts the
                      // charges of kOrderCells / sort_parts consecutive cells)
  int key_lv;         // levels of the order key: Morton index on a 2^key_lv grid (>= kOrderLevels;
                      // finer than the 16^3 cells only for the far-field tree)
  long long chg;      // offset of this system's charges (xyz at 3*chg, q at chg, phi at chg)
  long long src;      // offset of its 2n real+Kelvin source records (real first)
  long long surf;     // offset of its M surface records
  long long coef;     // offset of its P = (p+1)^2 correction coefficients
  long long mn;       // offset of its p+1 Kirkwood coefficients M_n
  long long mom;      // index of its first moment row
  int mom_blocks;     // moment rows of this system (FP64 path: one per k_moments block; FP32
                      // path: one per tile of k_moment_units)
  int mom_tile;       // charges per moment row
  long long mzo;      // FP32 path: offset of its (p+1) x n moment tables (powers, weights)
  long long part;     // offset of its pair partials (n_chunks * n elements)
  int ncr, nck, ncs;  // source chunks: real, Kelvin, surface
  int chunk;          // sources per real/Kelvin chunk; FP32 path: also the targets per block of
                      // the pair kernel's real/Kelvin items (blocks and chunks coincide)
  int chunk_s;        // points per surface chunk
  int tb;             // targets per target block of the pair kernel's surface items (FP32 path:
                      // a warp's group, 32 K) and of every FP64 pair item
  int n_tb;           // such target blocks
  int k5_first;       // first reduce item of this system
  int k5_count;       // reduce items of this system
  float dc2;          // squared near distance of the FP32 pair-sum box test, (kNearRel a)^2
  long long sb;       // offset (8-byte slots) of its auxiliary-sphere solid-harmonic table (M x P)
  long long bb;       // first 32-record box of this system (real boxes, then Kelvin boxes)
  // double-float (hi, lo) constants of the FP32 path's record arithmetic (k_setup): k/eps1, a,
  // a^2, and q_K = q (qk1 r_K + qk0) with qk1 = (k/(eps1 a)) (gamma - dbar/2),
  // qk0 = (k/(eps1 a)) dbar R_tau / 2; rc2 = (2 kCentreRel a)^2 (FP32)
  float2 f_kc, f_a, f_a2, f_qk1, f_qk0;
  float f_rc2;
  // and of the FP32 moment inputs: 1/a, dbar/2, R_tau/a
  float2 f_inv_a, f_hdbar, f_Rt_a;
};

// Inputs of a build pass, in device memory: the charges' coordinates (3 per charge) and values,
// in input order.  With copy set they are the caller's device arrays, read by the pass itself
// (no separate copy launch), and k_order_keys also writes them to the engine's own arrays
// (xyz_own, q_own), which every later kernel reads; otherwise they are the engine's own arrays.
struct InDesc {
  const double* xyz;
  const double* q;
  int copy;
  int pad;
};

// Spatial order (k_order.cu): charges sorted by the Morton index of their cell on a 16^3 grid
// over [-a, a]^3 and, inside a cell, by their key (the Morton index on the finer 2^key_lv grid, the
// same as the cell's when key_lv = kOrderLevels) and their input index.  perm[chg + i] = input index of sorted position
// i (its inverse iperm is written by k_images).  Pair-sum records, pair partials and move work use sorted positions.
// launch_order writes the cell keys and the cell histogram (items = (system, block of
// kOrderBlock charges)), then sorts each system in sort_parts blocks (sitems = (system, part)),
// each taking a run of consecutive cells; its first kernel also zeroes the nreset counters at
// ctr_reset.  hist (kOrderCells ints per system, then one counter per system) must be zero on
// entry and is zero again on exit; scr is scratch of 2 ints per charge (used by a block whose
// cells hold more charges than its shared memory).
constexpr int kOrderLevels = 4;
constexpr int kOrderGrid = 1 << kOrderLevels;
constexpr int kOrderCells = kOrderGrid * kOrderGrid * kOrderGrid;
constexpr int kOrderBlock = 256;  // charges per k_order_keys / k_images work item
void init_order_kernels();  // one-time function attributes (call outside stream capture)
// Charges a k_order_sort block sorts in shared memory at most (more use the scratch buffer), and
// the per-launch capacity for an engine whose largest share of a sort block is max_n charges.
constexpr int kOrderSmemMaxN = 24576;
int order_smem_charges(int64_t max_n);
// Sort blocks for a system of n charges: about one per kSortPartCharges, a power of two up to
// kSortMaxParts (every block reads all n keys, so a few thousand charges per block).
constexpr int kSortPartCharges = 2048;
constexpr int kSortMaxParts = 128;
int order_sort_parts(int64_t n);
// xs (FP32 path, else null): 2 float4 per charge in input order, the (hi, lo) split of
// (x, y, z, q): xs[2 g] = hi parts, xs[2 g + 1] = lo parts.  status: kStOutside for a charge at
// |x| >= a or with a non-finite coordinate or charge.
void launch_order(const SysDev* sys, int nsys, const int2* items, int nitems, const int2* sitems, int nsitems,
                  const InDesc* in, double* xyz_own, double* q_own, int* key, int* hist, int* scr, int* perm,
                  float4* xs, int* status, unsigned int* ctr_reset, int nreset, int smem_n, cudaStream_t st);
// Boxes of 32 consecutive sorted records: a warp's targets and a box farther apart than
// kNearRel a use plain FP32 coordinates in the pair sum, nearer ones the hi/lo-split form.
constexpr int kBox = 32;
constexpr double kNearRel = 0.08;
// Largest block of the FP32 path's real and Kelvin items (charges; blocks and chunks coincide
// there, see k_pairs_f32.cuh): the pair kernel keeps one (hi, lo) sum per source of a chunk in
// shared memory per warp.
constexpr int kSymChunkMax = 512;

// Offsets of the surface-record and coefficient tables for one engine.
struct Tables {
  const double* rec_a;    // vertical recurrence coefficient a_nm, index n(n+1)/2 + m
  const double* rec_b;    // vertical recurrence coefficient b_nm
  const double* sect;     // sectoral factor sqrt((2m-1)/(2m)) (m >= 2), 1 for m = 1
  const double* inv_np1;  // 1/(n+1), for the Legendre recurrence
  const float2* rec_a2;   // the same three tables as double-float pairs (hi, lo)
  const float2* rec_b2;
  const float2* sect2;
  const float2* leg_a2;   // Legendre recurrence (2n+1)/(n+1) and n/(n+1), n <= pmax, as (hi, lo)
  const float2* leg_b2;   // (stored after sect2 in the same array)
  const double* sprod;    // sectoral normalisation prod_{k <= m} sect[k] (stored after sect)
  const float2* sprod2;   // the same as (hi, lo) (stored after leg_b2)
  const float2* mbeta2;   // rescaled column chain of k_moment_units: beta_nm (index n(n+1)/2 + m)
  const float2* mnrm2;    // and its factor e_nm sprod_m back to T_nm (k_setup)
  int pmax;
};

// ---- launchers (k_sources.cu) ----
void init_source_kernels();  // one-time function attributes (call outside stream capture)
// Parameter-only work, once per layout: derived scalars, M_n, recurrence tables and the
// Fibonacci points/weights of every system (written to surfx).
void launch_setup(SysDev* sys, int nsys, double* Mn, double* rec_a, double* rec_b, double* sect, double* inv_np1,
                  float2* rec_a2, float2* rec_b2, float2* sect2, float2* mtab, int pmax, dbl4* surfx,
                  cudaStream_t st);
constexpr int kCoefChunk = 32;  // coefficients per k_coef_reduce block
// Records at sorted positions (items = (system, block of kOrderBlock sorted positions)) and the
// inverse of the order (iperm: input index -> sorted position, for the move kernels); the FP32
// path also writes the boxes (2 float4 per box: min and max of the hi coordinates).
void launch_images(const SysDev* sys, const int2* items, int nitems, const double* xyz, const double* q,
                   const float4* xs, const int* perm, int* iperm, float4* src_hi, float4* src_lo, dbl4* src64,
                   float4* boxes, int prec, int* status, cudaStream_t st);
// Moment rows: per block, sum_i q_i (M_n - gamma - c_i) T_nm(x_i/a) for the P coefficients
// (slots 0 .. P-1) and the block's centre constant (slot P).
// G: charges per moment group (moment_smem_group; the layout's tiles are multiples of it).
void launch_moments(const SysDev* sys, const int2* items, int nitems, int maxP, int G, const InDesc* in,
                    const double* Mn, Tables tab, int prec, double* mom, int mom_stride, cudaStream_t st);
// FP32 path, in two kernels.  k_moment_prep (items = (system, block of kMomPrepCharges charges)):
// per charge its double-float moment inputs -- geo = (2w hi, 2w lo, rho^2 hi, rho^2 lo), the
// powers (u + i v)^m (mz, (re hi, re lo, im hi, im lo)) and the weights q (M_n - gamma - c)
// (mwq) for m, n = 0..p at mzo + (m or n) n_sys + i -- and its centre constant (mcen, FP64).
// k_moment_units (units = (system, tile << 7 | column pair j), one warp each): row mom + tile of
// the moments of the columns m = j and p - j over the tile's charges, and slot P (the centre
// constants) for j = 0.  A programmatic dependent of the prep; its dependent may start at its end.
constexpr int kMomPrepThreads = 128;
constexpr int kMomPrepSplit = 4;  // threads per charge
constexpr int kMomPrepCharges = kMomPrepThreads / kMomPrepSplit;
constexpr int kMomUnitWarps = 4;  // small blocks: the units of a launch spread evenly over the SMs
constexpr int kMomUnitSteps = 8;  // chain steps per warp reduction (16 values)
inline int moment_unit_pairs(int p) { return p / 2 + 1; }
// Slots of the beta_nm table (mbeta2): rows n <= pmax + kMomUnitSteps, so that a chain may step
// past its last degree inside a batch without a bounds test; the mnrm2 table follows it.
__host__ __device__ constexpr int moment_beta_slots(int pmax)
{
  return (pmax + 1 + kMomUnitSteps) * (pmax + 2 + kMomUnitSteps) / 2;
}
void launch_moment_prep(const SysDev* sys, const int2* items, int nitems, const InDesc* in, const double* Mn,
                        float4* geo, float4* mz, float2* mwq, double* mcen, cudaStream_t st);
void launch_moment_units(const SysDev* sys, const int2* units, int nunits, const float4* geo,
                         const float4* mz, const float2* mwq, const double* mcen, Tables tab, double* mom,
                         int mom_stride, cudaStream_t st);
int moment_smem_group(int maxP, int blocks_per_sm);
// Moments are stored in the moment arithmetic (FP64 path: double; FP32 path: FP32 (hi, lo)
// pairs), one 8-byte slot each; the coefficients as double (coef) and as (hi, lo) pairs (coef2).
void launch_coef_reduce(const SysDev* sys, const int2* items, int nitems, const double* mom, int mom_stride,
                        const double* Mn, double* coef, float2* coef2, double* r0, int prec, cudaStream_t st);
// Solid harmonics of the auxiliary-sphere points (once per layout; items = (system, point block)
// of one representative system per table).
void launch_surface_basis(const SysDev* sys, const int2* items, int nitems, Tables tab, const dbl4* surfx, double* sb,
                          int prec, cudaStream_t st);
// Surface records from the coefficients: with the basis table sb (a GEMV per point), or, when
// sb is null, by running the solid-harmonic recurrence at every point.
// pw: surface points per warp of k_surface_mat (1, 2 or 4; items of kSurfWarps pw points) when
// the basis table sb is given.
void launch_surface(const SysDev* sys, const int2* items, int nitems, int maxP, int pw, const double* coef,
                    const float2* coef2, const double* sb, Tables tab, float4* surf_a, float4* surf_b,
                    dbl4* surf64_a, double* surf64_b, dbl4* surfx, double2* surfqd, int prec, cudaStream_t st);
constexpr int kSurfPointsPerBlock = 8;  // points per block of k_surface and k_surface_basis
constexpr int kSurfMatWarps = 8;        // warps per block of k_surface_mat (1, 2 or 4 points each)
// Largest total size of the surface-basis tables of one engine; beyond it the surface step runs
// the recurrence at every point instead.
constexpr size_t kMaxSurfBasisBytes = size_t(4) << 30;
constexpr int kMomTile = 256;  // largest moment tile (charges per moment block)

// ---- launchers (k_pairs.cu) ----
struct PairConfig {
  int threads;         // CTA size
  int k;               // targets per thread
  int items_per_slot;  // pair items per resident CTA slot of the layout
};
int pair_config_count();
PairConfig pair_config(int idx);
int pair_workers_per_cta(int cfg);  // FP32 pair kernel: warps, each an independent worker
int pair_kernel_of(int cfg);  // kernel variant (threads, k) of a configuration
int pairs_f32_occupancy(int cfg);
int pairs_f32_block_regs(int cfg);  // registers a CTA of the configuration holds
int chain_block_regs(int prec);     // the same for the largest coefficient / surface CTA
int pairs_f64_occupancy();
constexpr int kF64TargetsPerBlock = 128;
constexpr int kReduceTargetsPerBlock = 32;
// Persistent pair-sum launches: each CTA takes items of w1 until it is exhausted, then of w2.
// pdl: launched as a programmatic dependent of the stream's previous kernel (the kernels wait
// for it before touching any work).
void launch_pairs_f32(int cfg, int grid, const SysDev* sys, PairWork w1, PairWork w2, const float4* src_hi,
                      const float4* src_lo, const float4* surf_a, const float4* surf_b, const float4* boxes,
                      float2* part, cudaStream_t st, bool pdl = false);
void launch_pairs_f64(int grid, const SysDev* sys, PairWork w1, PairWork w2, const dbl4* src64,
                      const dbl4* surf64_a, const double* surf64_b, double* part64, cudaStream_t st,
                      bool pdl = false);
// Reduce the pair partials of the launched items to potentials and energies; the energies of
// system sel[r] are summed from the launch items sel_rng[r] = (first, count), ranges ascending
// and contiguous; counter[r] (zero before the launch, zero after it) counts r's finished items.
// pdl: launched as a programmatic dependent of the pair kernel that precedes it in the stream.
// energy == nullptr: only the per-block energy terms (epart, two doubles per launch item) are
// written; the reader sums them (Engine::read_energies), which spares every block the fence and
// atomic of the last-block completion.
// Where a potential pass also writes its results for the caller, read by k_reduce from device
// memory (so that a captured graph serves any destination): the selected potential in input order
// (device memory, or pinned host memory), the per-block energy terms (pinned host memory) and the
// pass's status flags, one byte per flag bit (pinned host memory, zeroed by the host before the
// pass; bytes, so that blocks setting different flags never overwrite one another); null
// pointers: nowhere.
struct OutDesc {
  double* phi;
  double* epart;
  unsigned char* status;
  int what;  // 0 Coulomb, 1 reaction, 2 total
  int pad;
};
constexpr int kStBits = 4;  // status flag bits mirrored by OutDesc::status
void launch_reduce(const SysDev* sys, const int* sel, const int2* sel_rng, int nsel, const int2* items, int nitems,
                   const float2* part, const double* part64, int prec, const double* q, const int* perm,
                   const double* r0, double* phi_c, double* phi_r, double* phi_t, double* epart, double* energy,
                   unsigned int* counter, int* status, const OutDesc* out, cudaStream_t st, bool pdl = false);

// ---- fields (k_field.cu): potential and E = -grad phi in one pass over the pair items ----
int field_f32_occupancy(int cfg);
int field_f64_occupancy();
// FP32: two float4 per (chunk, target) slot, (hi, lo) of (phi, Ex, Ey, Ez); FP64: one dbl4.
// Work lists as for the pair kernels (w1, then w2).
void launch_field_f32(int cfg, int grid, const SysDev* sys, PairWork w1, PairWork w2, const float4* src_hi,
                      const float4* src_lo, const float4* surf_a, const float4* surf_b, const float4* boxes,
                      float4* fpart, cudaStream_t st, bool pdl = false);
void launch_field_f64(int grid, const SysDev* sys, PairWork w1, PairWork w2, const dbl4* src64,
                      const dbl4* surf64_a, const double* surf64_b, dbl4* fpart64, cudaStream_t st,
                      bool pdl = false);
// as launch_reduce, plus the Coulomb, reaction and total fields (3 doubles per charge, input order)
void launch_reduce_field(const SysDev* sys, const int* sel, const int2* sel_rng, int nsel, const int2* items,
                         int nitems, const float4* fpart, const dbl4* fpart64, int prec, const double* q,
                         const int* perm, const double* r0, double* phi_c, double* phi_r, double* phi_t,
                         double* E_c, double* E_r, double* E_t, double* epart, double* energy, unsigned int* counter,
                         int* status, cudaStream_t st);

// ---- single-charge moves (k_delta.cu) ----
// One request: move charge k of system sys to (x, y, z).
struct DeltaReq {
  int sys;
  int k;
  double x, y, z;
};
constexpr int kDeltaBlock = 256;  // rows / surface points per delta work item
void init_delta_kernels();
void launch_surface_potentials(const SysDev* sys, const int2* items, int nitems, const double* xyz, const double* q,
                               const dbl4* surfx, double2* vsurf, cudaStream_t st);
void launch_delta(const SysDev* sys, const int4* items, int nitems, const int2* req_items, const DeltaReq* reqs,
                  int nreq, const double* xyz, const double* q, const int* perm, const int* iperm,
                  const float4* src_hi, const float4* src_lo, const dbl4* src64, const dbl4* surfx,
                  const double2* surfqd, const double2* vsurf, const double* Mn, Tables tab, double* dpart,
                  double* de, unsigned int* counter, int* status, cudaStream_t st);
void launch_move(const SysDev* sys, const int2* surf_items, int n_surf_items, const DeltaReq* reqs, int nreq,
                 Tables tab, int maxP, double* xyz, const double* q, const double* Mn, double* coef, float2* coef2,
                 double* r0, const dbl4* surfx, double2* surfqd, double2* vsurf, int have_v, float4* surf_a,
                 float4* surf_b, dbl4* surf64_a, double* surf64_b, const int* iperm, float4* src_hi, float4* src_lo,
                 dbl4* src64, float4* boxes, cudaStream_t st);

}  // namespace hsma
