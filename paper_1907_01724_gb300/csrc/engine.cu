// Host engine and C ABI of the HSMA library.
//
// An Engine owns the device state of one or more independent cavity systems (a single
// hsma_t handle is an engine with one system).  It lays every system's arrays out in one
// device workspace, builds the work lists of the kernels (longest pair items first), and
// records the two device phases as CUDA graphs:
//   build:     moment rows (FP32 path: k_moment_prep -> k_moment_units; FP64 path: k_moments)
//              -> k_coef_reduce -> k_surface_mat, beside k_order_* -> k_images     (Sec. 2.3-2.4)
//   potential: k_pairs -> k_reduce                                     (Algorithm 1 step 5)
// or, for an evaluation right after a build, both in one graph (issue_fused).  Graphs are
// re-recorded whenever the layout (sizes, tile configuration, pair schedule) or workspace changes.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "engine.h"

namespace hsma {

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

int Engine::fail(int code, const char* fmt, ...)
{
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  err = buf;
  return code;
}

int Engine::cuda_fail(cudaError_t e, const char* what)
{
  cudaGetLastError();
  return fail(HSMA_E_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call)                                  \
  do {                                            \
    cudaError_t e_ = (call);                      \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

int Engine::init(int dev, void* user_stream, int precision)
{
  device = dev;
  prec = precision;
  CK(cudaSetDevice(device));
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
  num_sms = sms;
  if (user_stream) {
    stream = (cudaStream_t)user_stream;
    own_stream = false;
  } else {
    // work runs on a stream of our own (graph capture is not possible on the legacy stream),
    // ordered after and before the caller's legacy-stream work by events (enter/leave)
    CK(cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking));
    own_stream = true;
    CK(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
  }
  static bool attrs_done[64] = {false};
  if (device >= 0 && device < 64 && !attrs_done[device]) {
    init_source_kernels();
    init_order_kernels();
    init_delta_kernels();
    attrs_done[device] = true;
  }
  occ_f32.assign(pair_config_count(), 0);
  for (int c = 0; c < pair_config_count(); ++c) occ_f32[c] = pairs_f32_occupancy(c);
  occ_f64 = pairs_f64_occupancy();
  regs_f32.assign(pair_config_count(), 0);
  for (int c = 0; c < pair_config_count(); ++c) regs_f32[c] = pairs_f32_block_regs(c);
  chain_regs = chain_block_regs(prec);
  CK(cudaDeviceGetAttribute(&sm_regs, cudaDevAttrMaxRegistersPerMultiprocessor, device));
  occ_field.assign(pair_config_count(), 0);
  for (int c = 0; c < pair_config_count(); ++c) occ_field[c] = field_f32_occupancy(c);
  occ_field64 = field_f64_occupancy();
  CK(cudaEventCreate(&ev_pair0));
  CK(cudaEventCreate(&ev_tree0));
  CK(cudaEventCreate(&ev_tree1));
  CK(cudaEventCreate(&ev_pair1));
  CK(cudaEventCreate(&ev_pot1));
  CK(cudaEventCreate(&ev_tune0));
  CK(cudaEventCreate(&ev_tune1));
  CK(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
  {
    int least = 0, greatest = 0;
    CK(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    prio_hi = greatest;
    prio_mid = std::min(greatest + 1, least);
  }
  CK(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ev_join, cudaEventDisableTiming));
  CK(cudaEventCreateWithFlags(&ev_img, cudaEventDisableTiming));
  CK(cudaGetLastError());
  return HSMA_OK;
}

int& launch_priority()
{
  static thread_local int p = 0;
  return p;
}

void Engine::enter()
{
  if (own_stream) {
    cudaEventRecord(ev_in, cudaStreamLegacy);
    cudaStreamWaitEvent(stream, ev_in, 0);
  }
}

void Engine::leave()
{
  if (own_stream) {
    cudaEventRecord(ev_out, stream);
    cudaStreamWaitEvent(cudaStreamLegacy, ev_out, 0);
  }
}

int Engine::last_pot_time(float* ms)
{
  if (!pair_timed) return fail(HSMA_E_STATE, "no pair sum has run");
  CK(cudaStreamSynchronize(stream));
  CK(cudaEventElapsedTime(ms, ev_pair0, ev_pot1));
  return HSMA_OK;
}

int Engine::last_pair_time(float* ms)
{
  if (!pair_timed) return fail(HSMA_E_STATE, "no pair sum has run");
  CK(cudaStreamSynchronize(stream));
  CK(cudaEventElapsedTime(ms, ev_pair0, ev_pair1));
  return HSMA_OK;
}

Engine::~Engine()
{
  if (device >= 0) cudaSetDevice(device);
  drop_graphs();
  if (ws_owned && ws) cudaFree(ws);
  if (energy_h) cudaFreeHost(energy_h);
  if (host_stage) cudaFreeHost(host_stage);
  if (fpart_d) cudaFree(fpart_d);
  if (E_d) cudaFree(E_d);
  if (ev_pair0) cudaEventDestroy(ev_pair0);
  if (ev_tree0) cudaEventDestroy(ev_tree0);
  if (ev_tree1) cudaEventDestroy(ev_tree1);
  if (ev_pair1) cudaEventDestroy(ev_pair1);
  if (ev_pot1) cudaEventDestroy(ev_pot1);
  if (ev_tune0) cudaEventDestroy(ev_tune0);
  if (ev_tune1) cudaEventDestroy(ev_tune1);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  if (ev_img) cudaEventDestroy(ev_img);
  if (side) cudaStreamDestroy(side);
  if (ev_in) cudaEventDestroy(ev_in);
  if (ev_out) cudaEventDestroy(ev_out);
  if (own_stream && stream) cudaStreamDestroy(stream);
}

void Engine::drop_graphs()
{
  if (g_build) cudaGraphExecDestroy(g_build);
  if (g_pot) cudaGraphExecDestroy(g_pot);
  if (g_field) cudaGraphExecDestroy(g_field);
  if (g_fused) cudaGraphExecDestroy(g_fused);
  if (g_field_fused) cudaGraphExecDestroy(g_field_fused);
  g_build = g_pot = g_field = g_fused = g_field_fused = nullptr;
}

// ---------------------------------------------------------------------------------------
Layout Engine::make_layout(const std::vector<int64_t>& ns, int cfg) const
{
  Layout L;
  const int nsys = (int)spec.size();
  L.cfg = cfg;
  // TB: targets per pair item (FP64) or per surface item of the FP32 pair kernel (a warp's
  // group); TBf: targets per item of the FP32 field kernel (its CTA's targets)
  int TB, TBf, occ, nw;
  if (prec == HSMA_FP64) {
    TB = TBf = kF64TargetsPerBlock;
    occ = occ_f64 > 0 ? occ_f64 : 1;
    nw = 1;
  } else {
    const PairConfig pc = pair_config(cfg);
    TB = 32 * pc.k;
    TBf = pc.threads * pc.k;
    occ = occ_f32[cfg] > 0 ? occ_f32[cfg] : 1;
    nw = pair_workers_per_cta(cfg);
  }
  const int slots = num_sms * occ;
  // pair items wanted over the whole engine: a few per worker (CTA on the FP64 path, warp on the
  // FP32 path)
  const double desired = (prec == HSMA_FP64 ? 4.0 : (double)pair_config(cfg).items_per_slot) * slots * nw;
  // the pair items and moment blocks of the whole engine are apportioned by each system's share
  // of the work, so a batch of many small systems gets few, larger items per system
  double W = 0.0;
  int64_t totn_all = 0;
  int maxP_all = 1;
  for (int s = 0; s < nsys; ++s) {
    W += (double)ns[s] * (2.0 * ns[s] + 1.3 * spec[s].M);
    totn_all += ns[s];
    maxP_all = std::max(maxP_all, (spec[s].p + 1) * (spec[s].p + 1));
  }
  // FP64 path (k_moments): charges per moment group, the largest group when the moment blocks
  // fit in about one wave, half-size shared memory (two blocks per SM) when there are many waves
  int G = moment_smem_group(maxP_all, 1);
  if (totn_all > 4 * (int64_t)num_sms * G) G = moment_smem_group(maxP_all, 2);
  L.momG = G;
  // FP32 moment units (k_moment_units): a warp per (tile of kg groups of 32 charges, column
  // pair), kg chosen so that a launch has about 96 units per SM (a few per resident warp) or,
  // for small engines, one group per tile
  int kg = 1;
  if (prec != HSMA_FP64) {
    int64_t U1 = 0;
    for (int s = 0; s < nsys; ++s) U1 += (ns[s] + 31) / 32 * moment_unit_pairs(spec[s].p);
    kg = (int)std::max<int64_t>(1, U1 / (96 * (int64_t)num_sms));
  }
  // the far-field tree replaces the direct real/Kelvin pair sum of a single FP32 system
  L.tree = prec != HSMA_FP64 && far_theta > 0.0 && nsys == 1 && ns[0] > 0;
  if (L.tree) {
    L.tL = tree_levels(ns[0]);
    L.tP = far_order;
  }
  L.sd.resize(nsys);
  int64_t zoff = 0;
  int64_t chg = 0, surf = 0, coef = 0, mn = 0, mom = 0, part = 0, boxes = 0;
  int k5 = 0;
  L.maxP = 1;
  L.pmax = 0;
  for (int s = 0; s < nsys; ++s) {
    const SysSpec& sp = spec[s];
    SysDev d;
    memset(&d, 0, sizeof(d));
    const int64_t n = ns[s];
    d.a = sp.a; d.eps1 = sp.eps1; d.eps2 = sp.eps2; d.kappa = sp.kappa; d.tau = sp.tau; d.dy_rel = sp.dy_rel;
    d.coulk = sp.coulk;
    d.p = sp.p; d.P = (sp.p + 1) * (sp.p + 1); d.M = sp.M; d.F1 = sp.F1; d.F2 = sp.F2;
    d.n = (int)n;
    d.prec = prec;
    d.sort_parts = order_sort_parts(n);
    d.key_lv = L.tree ? std::max(kOrderLevels, L.tL) : kOrderLevels;
    d.chg = chg; d.src = 2 * chg; d.surf = surf; d.coef = coef; d.mn = mn;
    d.mom = mom;
    // FP64 path: charges per moment block, enough blocks to cover the SMs twice over the whole
    // engine, a multiple of the moment group G (charges whose solid harmonics a block forms at
    // once); FP32 path: kg groups of 32 charges per moment row
    if (prec != HSMA_FP64) {
      d.mom_tile = 32 * kg;
    } else {
      const double share = (double)n / std::max<double>((double)totn_all, 1.0);
      const int64_t want_blocks = std::max<int64_t>(1, (int64_t)std::llround(2.0 * num_sms * share));
      int64_t tile = (n + want_blocks - 1) / want_blocks;
      tile = std::max<int64_t>(G, tile / G * G);
      tile = std::min<int64_t>(tile, std::max(G, kMomTile / G * G));
      d.mom_tile = (int)tile;
    }
    d.mom_blocks = (int)((n + d.mom_tile - 1) / d.mom_tile);
    d.mzo = zoff;  // FP32 path (zoff advances with the unit items below)
    d.tb = TB;
    d.n_tb = (int)((n + TB - 1) / TB);
    if (n > 0) {
      const double Ws = (double)n * (2.0 * n + 1.3 * sp.M);
      const double items_s = std::max(1.0, std::round(desired * Ws / std::max(W, 1.0)));
      if (prec == HSMA_FP64) {
        const int64_t chunks_total = std::max<int64_t>(1, (int64_t)std::ceil(items_s / d.n_tb));
        const int64_t per = (2 * n + sp.M + chunks_total - 1) / chunks_total;
        const int unit = kF64TargetsPerBlock;
        int64_t chunk = std::max<int64_t>(per, unit);
        chunk = (chunk + unit - 1) / unit * unit;
        d.chunk = (int)chunk;
        d.chunk_s = (int)chunk;
        d.ncr = (int)((n + chunk - 1) / chunk);
        d.nck = d.ncr;
        d.ncs = (int)((sp.M + chunk - 1) / chunk);
      } else {
        // real and Kelvin: nb blocks that are also the chunks, nb (nb + 1) items (each unordered
        // pair of blocks once, real and Kelvin); a block is a whole number of the pair kernel's
        // target groups and at most kSymChunkMax charges
        const double items_rk = L.tree ? 0.0 : items_s * (2.0 * n) / (2.0 * n + 1.3 * sp.M);
        if (L.tree) {
          // kTreeRootSplit chunks each: the tree's real and Kelvin sums (k_tree_eval), no pair items
          d.chunk = (int)n;
          d.ncr = d.nck = kTreeRootSplit;
        } else {
          const int64_t nb = std::max<int64_t>(1, (int64_t)std::floor(std::sqrt(std::max(items_rk, 1.0))));
          int64_t chunk = (n + nb - 1) / nb;
          chunk = (chunk + TB - 1) / TB * TB;
          chunk = std::min<int64_t>(std::max<int64_t>(chunk, TB), kSymChunkMax / TB * TB);
          d.chunk = (int)chunk;
          d.ncr = (int)((n + chunk - 1) / chunk);
          d.nck = d.ncr;
        }
        // surface: the rest of the items over the target groups, chunks of whole 32-point boxes
        const double items_sf = std::max(1.0, items_s - items_rk);
        const int64_t ncs_want = std::max<int64_t>(1, std::llround(items_sf / d.n_tb));
        int64_t chunk_s = (sp.M + ncs_want - 1) / ncs_want;
        chunk_s = std::max<int64_t>(kBox, (chunk_s + kBox - 1) / kBox * kBox);
        d.chunk_s = (int)chunk_s;
        d.ncs = (int)((sp.M + chunk_s - 1) / chunk_s);
      }
    }
    d.part = part;
    d.dc2 = (float)((kNearRel * sp.a) * (kNearRel * sp.a));
    d.bb = boxes;
    d.k5_first = k5;
    d.k5_count = (int)((n + kReduceTargetsPerBlock - 1) / kReduceTargetsPerBlock);
    L.sd[s] = d;
    if (prec == HSMA_FP64) {
      for (int b = 0; b < d.mom_blocks; ++b) L.it12.push_back(make_int2(s, b));
    } else {
      for (int b = 0; b < (int)((n + kMomPrepCharges - 1) / kMomPrepCharges); ++b) L.it12.push_back(make_int2(s, b));
      // (tiles < 2^24 for n <= 2^29 charges, pairs <= HSMA_P_MAX/2 + 1 < 2^7: fits an int)
      for (int t = 0; t < d.mom_blocks; ++t)
        for (int j = 0; j < moment_unit_pairs(sp.p); ++j) L.itmu.push_back(make_int2(s, (t << 7) | j));
      zoff += (int64_t)(sp.p + 1) * n;
    }
    for (int c = 0; c < (d.P + kCoefChunk - 1) / kCoefChunk; ++c) L.it2r.push_back(make_int2(s, c));
    for (int b = 0; b < (sp.M + kSurfPointsPerBlock - 1) / kSurfPointsPerBlock; ++b) L.it3.push_back(make_int2(s, b));
    for (int b = 0; b < d.k5_count; ++b) L.it5.push_back(make_int2(s, b));
    for (int b = 0; b < (int)((n + kOrderBlock - 1) / kOrderBlock); ++b) L.itord.push_back(make_int2(s, b));
    for (int b = 0; b < d.sort_parts; ++b) L.itsort.push_back(make_int2(s, b));
    const int nch = d.ncr + d.nck + d.ncs;
    if (prec == HSMA_FP64) {
      for (int tb = 0; tb < d.n_tb; ++tb)
        for (int c = 0; c < nch; ++c) L.it4.push_back(make_int4(s, tb, c, 0));
    } else if (n > 0) {
      // the pair kernel: each unordered pair of real/Kelvin blocks once (none with the tree),
      // surface items per group
      for (int b = 0; b < (L.tree ? 0 : d.ncr); ++b)
        for (int c = b; c < d.ncr; ++c) {
          L.it4.push_back(make_int4(s, b, c, 0));
          L.it4.push_back(make_int4(s, b, d.ncr + c, 0));
        }
      for (int tb = 0; tb < d.n_tb; ++tb)
        for (int c = d.ncr + d.nck; c < nch; ++c) L.it4.push_back(make_int4(s, tb, c, 0));
      // the field kernel: every (target block, chunk) one way (no field pass with the tree)
      const int ntbf = L.tree ? 0 : (int)((n + TBf - 1) / TBf);
      for (int tb = 0; tb < ntbf; ++tb)
        for (int c = 0; c < nch; ++c) L.it4f.push_back(make_int4(s, tb, c, 0));
    }
    chg += n;
    surf += sp.M;
    coef += d.P;
    mn += sp.p + 1;
    mom += d.mom_blocks;
    part += (int64_t)nch * n;
    boxes += 2 * ((n + kBox - 1) / kBox);
    k5 += d.k5_count;
    L.maxP = std::max(L.maxP, d.P);
    L.pmax = std::max(L.pmax, sp.p);
  }
  // auxiliary-sphere solid-harmonic tables, one per distinct (tau, M, F1, F2, p) (the table is
  // independent of a), built by a representative system
  {
    std::map<std::tuple<double, int, int, int, int>, int64_t> groups;
    int64_t off_sb = 0;
    for (int s = 0; s < nsys; ++s) {
      const SysSpec& sp = spec[s];
      const auto key = std::make_tuple(sp.tau, sp.M, sp.F1, sp.F2, sp.p);
      auto f = groups.find(key);
      if (f == groups.end()) {
        f = groups.emplace(key, off_sb).first;
        off_sb += (int64_t)sp.M * L.sd[s].P;
        for (int b = 0; b < (sp.M + kSurfPointsPerBlock - 1) / kSurfPointsPerBlock; ++b)
          L.itsb.push_back(make_int2(s, b));
      }
      L.sd[s].sb = f->second;
    }
    L.totSB = off_sb;
    L.use_sb = 8 * (size_t)off_sb <= kMaxSurfBasisBytes;
    if (!L.use_sb) L.itsb.clear();
    // with the basis, the per-step surface kernel takes surf_pw points per warp: as many as keep
    // at least four blocks per SM (fewer, larger blocks amortise the coefficient staging; more
    // blocks finish sooner when the launch is short of them)
    if (L.use_sb) {
      int64_t totM = 0;
      for (int s = 0; s < nsys; ++s) totM += spec[s].M;
      L.surf_pw = 1;
      for (int pw : {4, 2})
        if (totM / (kSurfMatWarps * pw) >= 4 * (int64_t)num_sms) {
          L.surf_pw = pw;
          break;
        }
      const int pts = kSurfMatWarps * L.surf_pw;
      for (int s = 0; s < nsys; ++s)
        for (int b = 0; b < (spec[s].M + pts - 1) / pts; ++b) L.it3m.push_back(make_int2(s, b));
    }
  }
  // longest pair items first (cost ~ targets x sources x per-source weight); among real/Kelvin
  // items of equal cost, the blocks nearest each other first: charges are in spatial order, so
  // the block distance |c - b| tracks their separation, and near blocks take the slower forms
  // (more checked boxes, their close pairs in the exact form; 1.5-2x the time of a far pair of
  // blocks measured on GB300), so the far, fast ones are left for the end of a launch
  const bool sym = prec != HSMA_FP64;
  auto cost_of = [&](const int4& it, bool field) {
    const SysDev& d = L.sd[it.x];
    const bool rk = it.z < d.ncr + d.nck;
    const int cb = it.z < d.ncr ? it.z : it.z - d.ncr;
    int64_t nt, ns_, w = 10;
    if (sym && !field && rk) {
      // a real/Kelvin block against a chunk: both ways off the diagonal, one way on it (with
      // the self box checked)
      nt = std::min<int64_t>(d.chunk, d.n - (int64_t)it.y * d.chunk);
      w = 12;
    } else {
      const int64_t tbk = field ? TBf : d.tb;
      nt = std::min<int64_t>(tbk, d.n - (int64_t)it.y * tbk);
    }
    if (rk) {
      ns_ = std::min<int64_t>(d.chunk, d.n - (int64_t)cb * d.chunk);
    } else {
      ns_ = std::min<int64_t>(d.chunk_s, d.M - (int64_t)(it.z - d.ncr - d.nck) * d.chunk_s);
      w = 13;
    }
    return nt * ns_ * w;
  };
  auto is_rk = [&](const int4& it) { return it.z < L.sd[it.x].ncr + L.sd[it.x].nck; };
  for (auto& it : L.it4) it.w = 0;
  auto gap_of = [&](const int4& it) {
    const SysDev& d = L.sd[it.x];
    if (it.z >= d.ncr + d.nck) return 0;
    return std::abs((it.z < d.ncr ? it.z : it.z - d.ncr) - it.y);
  };
  std::stable_sort(L.it4.begin(), L.it4.end(), [&](const int4& x, const int4& y) {
    const int64_t cx = cost_of(x, false), cy = cost_of(y, false);
    return cx != cy ? cx > cy : gap_of(x) < gap_of(y);
  });
  // the overlapped pass launches the real/Kelvin items (which need only the records) apart from
  // the surface items (which wait for the coefficient chain)
  L.it4x = L.it4;
  L.nRK = (int)(std::stable_partition(L.it4x.begin(), L.it4x.end(), is_rk) - L.it4x.begin());
  // the field pass: on the FP64 path the same one-way list; on the FP32 path its own
  if (!sym) L.it4f = L.it4;
  for (auto& it : L.it4f) it.w = 0;
  std::stable_sort(L.it4f.begin(), L.it4f.end(),
                   [&](const int4& x, const int4& y) { return cost_of(x, true) > cost_of(y, true); });
  L.it4fx = L.it4f;
  L.nRKf = (int)(std::stable_partition(L.it4fx.begin(), L.it4fx.end(), is_rk) - L.it4fx.begin());
  {
    // a sort block's share: all of a one-block system, else twice the mean share of its blocks
    // (a denser run of cells spills to the scratch buffer)
    int64_t maxn = 0;
    for (const auto& d : L.sd)
      maxn = std::max<int64_t>(maxn, d.sort_parts == 1 ? d.n : (2 * (int64_t)d.n + d.sort_parts - 1) / d.sort_parts);
    L.order_smem_n = order_smem_charges(maxn);
  }
  L.totN = chg;
  L.totM = surf;
  L.totP = coef;
  L.totMn = mn;
  L.totMom = mom;
  L.totZ = zoff;
  L.totPart = part;
  L.totBoxes = boxes;
  L.mom_stride = (int)align_up((size_t)L.maxP + 1, 2);
  L.nw = nw;
  L.pair_grid = (int)std::max<size_t>(1, std::min<size_t>((L.it4.size() + nw - 1) / nw, (size_t)slots));

  // workspace plan
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + std::max<size_t>(bytes, 1), 256);
    return o;
  };
  const int ntri = (L.pmax + 1) * (L.pmax + 2) / 2;
  L.o_sys = take(sizeof(SysDev) * nsys);
  L.o_Mn = take(8 * L.totMn);
  L.o_rec_a = take(8 * (size_t)ntri);
  L.o_rec_b = take(8 * (size_t)ntri);
  L.o_sect = take(8 * 2 * (size_t)(L.pmax + 1));  // sect, then sprod
  L.o_inv_np1 = take(8 * (size_t)(L.pmax + 1));
  L.o_rec_a2 = take(8 * (size_t)ntri);
  L.o_rec_b2 = take(8 * (size_t)ntri);
  L.o_sect2 = take(8 * 4 * (size_t)(L.pmax + 1));  // sect2, the Legendre tables, sprod2
  L.o_mtab = take(8 * ((size_t)moment_beta_slots(L.pmax) + (size_t)ntri));
  L.o_xyz = take(24 * L.totN);
  L.o_q = take(8 * L.totN);
  if (prec == HSMA_FP64) {
    L.o_src64 = take(32 * 2 * L.totN);
    L.o_surf64a = take(32 * L.totM);
    L.o_surf64b = take(8 * L.totM);
    L.o_part64 = take(8 * L.totPart);
  } else {
    L.o_srchi = take(16 * 2 * L.totN);
    L.o_srclo = take(16 * 2 * L.totN);
    L.o_surfa = take(16 * L.totM);
    L.o_surfb = take(16 * L.totM);
    L.o_part = take(8 * L.totPart);
  }
  L.o_surfx = take(32 * L.totM);
  L.o_surfqd = take(16 * L.totM);
  L.o_vsurf = take(16 * L.totM);
  {
    int per_req = 1;
    for (const auto& d : L.sd)
      per_req = std::max(per_req, (d.n + kDeltaBlock - 1) / kDeltaBlock + (d.M + kDeltaBlock - 1) / kDeltaBlock);
    L.max_req = std::max(1, max_requests);
    L.ditem_cap = L.max_req * per_req;
    int surf_blocks = 1;
    for (const auto& d : L.sd) surf_blocks = std::max(surf_blocks, (d.M + kDeltaBlock - 1) / kDeltaBlock);
    L.mitem_cap = L.max_req * surf_blocks;
  }
  L.o_dreq = take(sizeof(DeltaReq) * (size_t)L.max_req);
  L.o_ditems = take(sizeof(int4) * (size_t)L.ditem_cap);
  L.o_dreqit = take(sizeof(int2) * (size_t)L.max_req);
  L.o_mitems = take(sizeof(int2) * (size_t)L.mitem_cap);
  L.o_dpart = take(8 * (size_t)L.ditem_cap);
  L.o_de = take(8 * (size_t)L.max_req);
  L.o_mom = take(8 * (size_t)L.totMom * L.mom_stride);
  if (prec != HSMA_FP64) {
    L.o_mgeo = take(16 * (size_t)L.totN);
    L.o_mz = take(16 * (size_t)L.totZ);
    L.o_mwq = take(8 * (size_t)L.totZ);
    L.o_mcen = take(8 * (size_t)L.totN);
    L.o_itmu = take(sizeof(int2) * L.itmu.size());
  }
  L.o_coef = take(8 * L.totP);
  L.o_coef2 = take(8 * L.totP);
  L.o_sb = take(L.use_sb ? 8 * (size_t)L.totSB : 0);
  L.o_itsb = take(sizeof(int2) * L.itsb.size());
  L.o_perm = take(4 * (size_t)L.totN);
  L.o_iperm = take(4 * (size_t)L.totN);
  L.o_key = take(4 * (size_t)L.totN);
  L.o_hist = take(4 * (size_t)nsys * (kOrderCells + 1));
  L.o_sortscr = take(8 * (size_t)L.totN);
  L.o_xs = take(prec == HSMA_FP64 ? 0 : 32 * (size_t)L.totN);
  L.o_boxes = take(2 * sizeof(float4) * (size_t)L.totBoxes);
  L.o_itord = take(sizeof(int2) * L.itord.size());
  L.o_itsort = take(sizeof(int2) * L.itsort.size());
  L.o_r0 = take(8 * (size_t)nsys);
  L.o_phic = take(8 * L.totN);
  L.o_phir = take(8 * L.totN);
  L.o_phit = take(8 * L.totN);
  L.o_epart = take(16 * L.it5.size());
  L.o_energy = take(16 * (size_t)nsys);
  L.o_ctr = take(16);
  L.o_outdesc = take(sizeof(OutDesc));
  L.o_indesc = take(sizeof(InDesc));
  L.o_redctr = take(4 * (size_t)nsys);
  L.o_it12 = take(sizeof(int2) * L.it12.size());
  L.o_it2r = take(sizeof(int2) * L.it2r.size());
  L.o_it3 = take(sizeof(int2) * L.it3.size());
  L.o_it3m = take(sizeof(int2) * L.it3m.size());
  L.o_it5 = take(sizeof(int2) * L.it5.size());
  L.o_it4 = take(sizeof(int4) * L.it4.size());
  L.o_it4x = take(sizeof(int4) * L.it4x.size());
  L.o_it4f = take(sizeof(int4) * L.it4f.size());
  L.o_it4fx = take(sizeof(int4) * L.it4fx.size());
  L.sel.resize(nsys);
  L.selrng.resize(nsys);
  for (int s = 0; s < nsys; ++s) {
    L.sel[s] = s;
    L.selrng[s] = make_int2(L.sd[s].k5_first, L.sd[s].k5_count);
  }
  L.o_sel = take(sizeof(int) * (size_t)nsys);
  L.o_selrng = take(sizeof(int2) * (size_t)nsys);
  if (L.tree) {
    const size_t nodes = (size_t)tree_node_count(L.tL), nm = (size_t)tree_nm(L.tP);
    L.o_tnode = take(sizeof(int2) * nodes);
    L.o_tgeo = take(sizeof(float4) * 2 * nodes);
    L.o_tbox = take(sizeof(float4) * 4 * nodes);
    L.o_tmom = take(sizeof(float2) * 2 * nodes * nm);
    L.o_tfarp = take(sizeof(float2) * kFarBlocks * (size_t)tree_nm(kFarOrder));
    L.o_tfarL = take(sizeof(float2) * (size_t)tree_nm(kFarOrder));
    L.o_tctr = take(16);
  }
  L.bytes = off;
  return L;
}

void Engine::carve()
{
  char* b = ws;
  sys_d = (SysDev*)(b + L.o_sys);
  Mn_d = (double*)(b + L.o_Mn);
  rec_a_d = (double*)(b + L.o_rec_a);
  rec_b_d = (double*)(b + L.o_rec_b);
  sect_d = (double*)(b + L.o_sect);
  inv_np1_d = (double*)(b + L.o_inv_np1);
  rec_a2_d = (float2*)(b + L.o_rec_a2);
  rec_b2_d = (float2*)(b + L.o_rec_b2);
  sect2_d = (float2*)(b + L.o_sect2);
  mtab_d = (float2*)(b + L.o_mtab);
  xyz_d = (double*)(b + L.o_xyz);
  q_d = (double*)(b + L.o_q);
  if (prec == HSMA_FP64) {
    src64_d = (dbl4*)(b + L.o_src64);
    surf64a_d = (dbl4*)(b + L.o_surf64a);
    surf64b_d = (double*)(b + L.o_surf64b);
    part64_d = (double*)(b + L.o_part64);
    srchi_d = srclo_d = surfa_d = surfb_d = nullptr;
    part_d = nullptr;
  } else {
    srchi_d = (float4*)(b + L.o_srchi);
    srclo_d = (float4*)(b + L.o_srclo);
    surfa_d = (float4*)(b + L.o_surfa);
    surfb_d = (float4*)(b + L.o_surfb);
    part_d = (float2*)(b + L.o_part);
    src64_d = nullptr;
    surf64a_d = nullptr;
    surf64b_d = nullptr;
    part64_d = nullptr;
  }
  surfx_d = (dbl4*)(b + L.o_surfx);
  surfqd_d = (double2*)(b + L.o_surfqd);
  vsurf_d = (double2*)(b + L.o_vsurf);
  dreq_d = (DeltaReq*)(b + L.o_dreq);
  ditems_d = (int4*)(b + L.o_ditems);
  dreqit_d = (int2*)(b + L.o_dreqit);
  mitems_d = (int2*)(b + L.o_mitems);
  dpart_d = (double*)(b + L.o_dpart);
  de_d = (double*)(b + L.o_de);
  mom_d = (double*)(b + L.o_mom);
  if (prec != HSMA_FP64) {
    mgeo_d = (float4*)(b + L.o_mgeo);
    mz_d = (float4*)(b + L.o_mz);
    mwq_d = (float2*)(b + L.o_mwq);
    mcen_d = (double*)(b + L.o_mcen);
    itmu_d = (int2*)(b + L.o_itmu);
  } else {
    mgeo_d = mz_d = nullptr;
    mwq_d = nullptr;
    mcen_d = nullptr;
    itmu_d = nullptr;
  }
  coef_d = (double*)(b + L.o_coef);
  coef2_d = (float2*)(b + L.o_coef2);
  sb_d = L.use_sb ? (double*)(b + L.o_sb) : nullptr;
  itsb_d = (int2*)(b + L.o_itsb);
  perm_d = (int*)(b + L.o_perm);
  iperm_d = (int*)(b + L.o_iperm);
  key_d = (int*)(b + L.o_key);
  hist_d = (int*)(b + L.o_hist);
  sortscr_d = (int*)(b + L.o_sortscr);
  xs_d = prec == HSMA_FP64 ? nullptr : (float4*)(b + L.o_xs);
  boxes_d = (float4*)(b + L.o_boxes);
  itord_d = (int2*)(b + L.o_itord);
  itsort_d = (int2*)(b + L.o_itsort);
  r0_d = (double*)(b + L.o_r0);
  phic_d = (double*)(b + L.o_phic);
  phir_d = (double*)(b + L.o_phir);
  phit_d = (double*)(b + L.o_phit);
  epart_d = (double*)(b + L.o_epart);
  energy_d = (double*)(b + L.o_energy);
  unsigned int* ctr = (unsigned int*)(b + L.o_ctr);
  ctr_pairs_d = ctr;
  ctr_red_d = (unsigned int*)(b + L.o_redctr);
  status_d = (int*)(ctr + 2);
  outdesc_d = (OutDesc*)(b + L.o_outdesc);
  indesc_d = (InDesc*)(b + L.o_indesc);
  in_loaded = false;
  ctr_delta_d = ctr + 3;
  it12_d = (int2*)(b + L.o_it12);
  it2r_d = (int2*)(b + L.o_it2r);
  it3_d = (int2*)(b + L.o_it3);
  it3m_d = (int2*)(b + L.o_it3m);
  it5_d = (int2*)(b + L.o_it5);
  it4_d = (int4*)(b + L.o_it4);
  it4x_d = (int4*)(b + L.o_it4x);
  it4f_d = (int4*)(b + L.o_it4f);
  it4fx_d = (int4*)(b + L.o_it4fx);
  ctr_pairs2_d = ctr + 1;
  sel_d = (int*)(b + L.o_sel);
  selrng_d = (int2*)(b + L.o_selrng);
}

int Engine::attach(void* ptr, size_t bytes)
{
  CK(cudaSetDevice(device));
  if (ptr && ((uintptr_t)ptr % 256) != 0) return fail(HSMA_E_INVALID_ARG, "workspace must be 256-byte aligned");
  CK(cudaStreamSynchronize(stream));
  if (ws_owned && ws) cudaFree(ws);
  ws = (char*)ptr;
  ws_cap = ptr ? bytes : 0;
  ws_owned = false;
  ws_user = ptr != nullptr;
  layout_uploaded = false;
  sources_ready = pot_ready = false;
  build_pending = false;
  drop_graphs();
  return HSMA_OK;
}

int Engine::set_sizes(const std::vector<int64_t>& ns)
{
  if (have_layout && ns == cur_ns && layout_uploaded) return HSMA_OK;
  const int cfg = prec == HSMA_FP64 ? 0 : choose_config(ns);
  L = make_layout(ns, cfg);
  rk_side = prec == HSMA_FP64 ? 1 : choose_side(ns);
  cur_ns = ns;
  have_layout = true;
  if (L.bytes > ws_cap) {
    if (ws_user) return fail(HSMA_E_OOM, "attached workspace has %zu bytes, %zu needed", ws_cap, L.bytes);
    CK(cudaStreamSynchronize(stream));
    if (ws) cudaFree(ws);
    ws = nullptr;
    ws_cap = 0;
    const size_t want = L.bytes + L.bytes / 4;
    cudaError_t e = cudaMalloc((void**)&ws, want);
    if (e != cudaSuccess) {
      cudaGetLastError();
      ws = nullptr;
      return fail(HSMA_E_OOM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    ws_cap = want;
    ws_owned = true;
  }
  carve();
  drop_graphs();
  CK(cudaMemcpyAsync(sys_d, L.sd.data(), sizeof(SysDev) * L.sd.size(), cudaMemcpyHostToDevice, stream));
  if (!L.it12.empty())
    CK(cudaMemcpyAsync(it12_d, L.it12.data(), sizeof(int2) * L.it12.size(), cudaMemcpyHostToDevice, stream));
  if (!L.itmu.empty())
    CK(cudaMemcpyAsync(itmu_d, L.itmu.data(), sizeof(int2) * L.itmu.size(), cudaMemcpyHostToDevice, stream));
  if (!L.it2r.empty())
    CK(cudaMemcpyAsync(it2r_d, L.it2r.data(), sizeof(int2) * L.it2r.size(), cudaMemcpyHostToDevice, stream));
  if (!L.it3.empty())
    CK(cudaMemcpyAsync(it3_d, L.it3.data(), sizeof(int2) * L.it3.size(), cudaMemcpyHostToDevice, stream));
  if (!L.it3m.empty())
    CK(cudaMemcpyAsync(it3m_d, L.it3m.data(), sizeof(int2) * L.it3m.size(), cudaMemcpyHostToDevice, stream));
  if (!L.it5.empty())
    CK(cudaMemcpyAsync(it5_d, L.it5.data(), sizeof(int2) * L.it5.size(), cudaMemcpyHostToDevice, stream));
  if (!L.it4.empty())
    CK(cudaMemcpyAsync(it4_d, L.it4.data(), sizeof(int4) * L.it4.size(), cudaMemcpyHostToDevice, stream));
  if (!L.it4x.empty())
    CK(cudaMemcpyAsync(it4x_d, L.it4x.data(), sizeof(int4) * L.it4x.size(), cudaMemcpyHostToDevice, stream));
  if (!L.it4f.empty())
    CK(cudaMemcpyAsync(it4f_d, L.it4f.data(), sizeof(int4) * L.it4f.size(), cudaMemcpyHostToDevice, stream));
  if (!L.it4fx.empty())
    CK(cudaMemcpyAsync(it4fx_d, L.it4fx.data(), sizeof(int4) * L.it4fx.size(), cudaMemcpyHostToDevice, stream));
  if (!L.itsb.empty())
    CK(cudaMemcpyAsync(itsb_d, L.itsb.data(), sizeof(int2) * L.itsb.size(), cudaMemcpyHostToDevice, stream));
  if (!L.itord.empty())
    CK(cudaMemcpyAsync(itord_d, L.itord.data(), sizeof(int2) * L.itord.size(), cudaMemcpyHostToDevice, stream));
  if (!L.itsort.empty())
    CK(cudaMemcpyAsync(itsort_d, L.itsort.data(), sizeof(int2) * L.itsort.size(), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(sel_d, L.sel.data(), sizeof(int) * L.sel.size(), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(selrng_d, L.selrng.data(), sizeof(int2) * L.selrng.size(), cudaMemcpyHostToDevice, stream));
  CK(cudaMemsetAsync(ctr_pairs_d, 0, 16, stream));
  CK(cudaMemsetAsync(ctr_red_d, 0, 4 * L.sd.size(), stream));
  CK(cudaMemsetAsync(energy_d, 0, 16 * L.sd.size(), stream));
  CK(cudaMemsetAsync(hist_d, 0, 4 * L.sd.size() * (kOrderCells + 1), stream));
  CK(cudaMemsetAsync(outdesc_d, 0, sizeof(OutDesc), stream));
  out_cur = OutDesc{nullptr, nullptr, nullptr, 0, 0};
  // parameter-only quantities (scalars, M_n, tables, quadrature grid, surface basis), once per layout
  launch_setup(sys_d, (int)L.sd.size(), Mn_d, rec_a_d, rec_b_d, sect_d, inv_np1_d, rec_a2_d, rec_b2_d, sect2_d,
               mtab_d, L.pmax, surfx_d, stream);
  CK(cudaGetLastError());
  launches += 1;
  if (L.use_sb && !L.itsb.empty()) {
    launch_surface_basis(sys_d, itsb_d, (int)L.itsb.size(), tables(), surfx_d, sb_d, prec, stream);
    CK(cudaGetLastError());
    launches += 1;
  }
  CK(cudaStreamSynchronize(stream));
  layout_uploaded = true;
  sources_ready = pot_ready = false;
  build_pending = false;
  return HSMA_OK;
}

Tables Engine::tables() const
{
  Tables t;
  t.rec_a = rec_a_d;
  t.rec_b = rec_b_d;
  t.sect = sect_d;
  t.inv_np1 = inv_np1_d;
  t.rec_a2 = rec_a2_d;
  t.rec_b2 = rec_b2_d;
  t.sect2 = sect2_d;
  t.leg_a2 = sect2_d + (L.pmax + 1);
  t.leg_b2 = sect2_d + 2 * (L.pmax + 1);
  t.sprod = sect_d + (L.pmax + 1);
  t.sprod2 = sect2_d + 3 * (L.pmax + 1);
  t.mbeta2 = mtab_d;
  t.mnrm2 = mtab_d + moment_beta_slots(L.pmax);
  t.pmax = L.pmax;
  return t;
}

TreeView Engine::tree_view() const
{
  TreeView t{};
  char* b = ws;
  t.sys = sys_d;
  t.key = key_d;
  t.perm = perm_d;
  t.hi = srchi_d;
  t.lo = srclo_d;
  t.node = (int2*)(b + L.o_tnode);
  t.geo = (float4*)(b + L.o_tgeo);
  t.box = (float4*)(b + L.o_tbox);
  t.mom = (float2*)(b + L.o_tmom);
  t.farp = (float2*)(b + L.o_tfarp);
  t.farL = (float2*)(b + L.o_tfarL);
  t.ctr = (unsigned int*)(b + L.o_tctr);
  t.L = L.tL;
  t.key_lv = L.sd[0].key_lv;
  t.P = L.tP;
  t.cmin = (L.tP + 1) * (L.tP + 1) / 3;  // ~850 instructions per evaluation against ~16 per pair
  t.theta = (float)far_theta;
  t.log_eps = (float)(std::log(0.1) + (L.tP + 1) * std::log(far_theta > 0.0 ? far_theta : 0.5));
  const double a = spec[0].a;
  t.rfar2 = (float)((kFarImageRel * a) * (kFarImageRel * a));
  t.inv_a = (float)(1.0 / a);
  return t;
}

// The tree's build (after the records) and its evaluation, on stream st; the evaluation's
// device time is taken with ev_tree0 / ev_tree1.
void Engine::issue_tree(cudaStream_t st)
{
  const TreeView tv = tree_view();
  const int n = L.sd[0].n;
  launch_tree_build(tv, n, st);
  cudaEventRecordWithFlags(ev_tree0, st, cudaEventRecordExternal);
  launch_tree_eval(tv, n, part_d, st);
  cudaEventRecordWithFlags(ev_tree1, st, cudaEventRecordExternal);
  tree_timed = true;
}

int Engine::last_tree_time(float* ms)
{
  if (!tree_timed) return fail(HSMA_E_STATE, "no far-field tree evaluation has run");
  CK(cudaStreamSynchronize(stream));
  CK(cudaEventElapsedTime(ms, ev_tree0, ev_tree1));
  return HSMA_OK;
}

void Engine::issue_moments()
{
  if (prec == HSMA_FP64) {
    launch_moments(sys_d, it12_d, (int)L.it12.size(), L.maxP, L.momG, indesc_d, Mn_d, tables(), prec, mom_d,
                   L.mom_stride, stream);
    return;
  }
  launch_moment_prep(sys_d, it12_d, (int)L.it12.size(), indesc_d, Mn_d, mgeo_d, mz_d, mwq_d, mcen_d, stream);
  launch_moment_units(sys_d, itmu_d, (int)L.itmu.size(), mgeo_d, mz_d, mwq_d, mcen_d, tables(), mom_d,
                      L.mom_stride, stream);
}

void Engine::issue_build()
{
  // fork: the spatial order and the pair-sum records on the second stream, beside the
  // moments -> coefficients -> surface chain; both are joined before the build ends
  const int nsys = (int)L.sd.size();
  const bool order = !L.itord.empty();
  if (order) {
    cudaEventRecord(ev_fork, stream);
    cudaStreamWaitEvent(side, ev_fork, 0);
    PriorityScope ps(prio_hi);
    launch_order(sys_d, nsys, itord_d, (int)L.itord.size(), itsort_d, (int)L.itsort.size(), indesc_d, xyz_d, q_d,
                 key_d, hist_d, sortscr_d, perm_d, xs_d, status_d, nullptr, 0, L.order_smem_n, side);
    launch_images(sys_d, itord_d, (int)L.itord.size(), xyz_d, q_d, xs_d, perm_d, iperm_d, srchi_d, srclo_d, src64_d,
                  boxes_d, prec, status_d, side);
    cudaEventRecord(ev_join, side);
  }
  issue_moments();
  launch_coef_reduce(sys_d, it2r_d, (int)L.it2r.size(), mom_d, L.mom_stride, Mn_d, coef_d, coef2_d, r0_d, prec,
                     stream);
  launch_surface(sys_d, L.use_sb ? it3m_d : it3_d, (int)(L.use_sb ? L.it3m.size() : L.it3.size()), L.maxP,
                 L.surf_pw, coef_d, coef2_d, sb_d, tables(), surfa_d, surfb_d, surf64a_d, surf64b_d, surfx_d,
                 surfqd_d, prec, stream);
  if (order) cudaStreamWaitEvent(stream, ev_join, 0);
}

int Engine::build_launch_count() const
{
  // order: 2 kernels (k_order_keys, k_order_sort) and k_images
  return (L.itord.empty() ? 0 : 3) + (L.it12.empty() ? 0 : 1) + (L.itmu.empty() ? 0 : 1) +
         (L.it2r.empty() ? 0 : 1) + (L.it3.empty() ? 0 : 1);
}

void Engine::issue_pot()
{
  const int nsys = (int)L.sd.size();
  if (L.tree) issue_tree(stream);
  cudaMemsetAsync(ctr_pairs_d, 0, sizeof(unsigned int), stream);
  if (!L.it4.empty()) {
    cudaEventRecordWithFlags(ev_pair0, stream, cudaEventRecordExternal);
    const int nit = (int)L.it4.size();
    const PairWork all{it4_d, nit, ctr_pairs_d, std::min(L.pair_grid * L.nw, nit)}, none{nullptr, 0, nullptr, 0};
    if (prec == HSMA_FP64)
      launch_pairs_f64(L.pair_grid, sys_d, all, none, src64_d, surf64a_d, surf64b_d, part64_d, stream);
    else
      launch_pairs_f32(L.cfg, L.pair_grid, sys_d, all, none, srchi_d, srclo_d, surfa_d, surfb_d, boxes_d, part_d,
                       stream);
    cudaEventRecordWithFlags(ev_pair1, stream, cudaEventRecordExternal);
  }
  launch_reduce(sys_d, sel_d, selrng_d, nsys, it5_d, (int)L.it5.size(), part_d, part64_d, prec, q_d, perm_d, r0_d,
                phic_d, phir_d, phit_d, epart_d, nullptr, ctr_red_d, status_d, outdesc_d, stream);
  if (!L.it4.empty()) cudaEventRecordWithFlags(ev_pot1, stream, cudaEventRecordExternal);
}

int Engine::pot_launch_count() const
{
  return (L.it4.empty() ? 0 : 1) + (L.it5.empty() ? 0 : 1) + (L.tree ? tree_launch_count() : 0);
}

// k_tree_marks, k_tree_leaf, k_tree_up per level below L, k_tree_far, k_tree_eval
int Engine::tree_launch_count() const { return 4 + (L.tL - kTreeTop); }

void Engine::launch_pair_items(PairWork w1, PairWork w2, int grid, cudaStream_t st, bool pdl)
{
  if (w1.nitems <= 0 && w2.nitems <= 0) return;
  if (prec == HSMA_FP64)
    launch_pairs_f64(grid, sys_d, w1, w2, src64_d, surf64a_d, surf64b_d, part64_d, st, pdl);
  else
    launch_pairs_f32(L.cfg, grid, sys_d, w1, w2, srchi_d, srclo_d, surfa_d, surfb_d, boxes_d, part_d, st, pdl);
}

// Build and potentials in one graph: the order and the records on the second stream beside the
// moment -> coefficient -> surface chain, then the pair sum and the reduction.  The real/Kelvin
// pair items need only the records; where they run is the layout's schedule (rk_side):
//   1: side:  k_order_keys -> k_order_sort -> k_images -> k_pairs (real/Kelvin, all CTA slots but
//             one per SM, lowest launch priority)
//      main:  k_moment_prep -> k_moment_units -> k_coef_reduce -> k_surface_mat -> k_pairs
//             (surface items, then the real/Kelvin items the first launch has not taken) -> join
//             -> k_reduce
//   2: as 1, with fewer CTAs in the side launch (side_ctas_per_sm)
//   0: side:  k_order_keys -> k_order_sort -> k_images
//      main:  the same chain -> [wait records] k_pairs (surface items, then every real/Kelvin
//             item) -> k_reduce
// With 1 the real/Kelvin sum fills the SMs that the chain's latency-bound kernels leave idle,
// but its persistent CTAs hold their SMs' registers until the real/Kelvin items run out, so the
// launch leaves one CTA slot per SM for the coefficient and surface kernels; still, these may
// wait for the whole real/Kelvin sum: (1) is faster for one or two cavities (0.326 against 0.349
// ms at N = 20000; 66 against 72 us for two cavities of N = 2000), (0) for a batch of 512 (6.2
// against 7.1 ms).  The autotuner times both for a size class.
// Either way each item is evaluated once, from the same lists and work counters, so results are
// bitwise the same.
void Engine::issue_fused()
{
  if (L.itord.empty()) {
    issue_build();
    issue_pot();
    return;
  }
  const int nsys = (int)L.sd.size();
  const int nS = (int)L.it4x.size() - L.nRK;
  const int occ = prec == HSMA_FP64 ? std::max(occ_f64, 1) : std::max(occ_f32[L.cfg], 1);
  const int slots = num_sms * occ;
  const int nw = L.nw;  // workers per CTA
  const bool side_rk = rk_side != 0 && L.nRK > 0;
  const int grid_rk = std::max(1, std::min((L.nRK + nw - 1) / nw, num_sms * side_ctas_per_sm(occ)));
  const int grid_s = std::max(1, std::min((nS + L.nRK + nw - 1) / nw, slots));
  cudaEventRecord(ev_fork, stream);
  cudaStreamWaitEvent(side, ev_fork, 0);
  // launch priorities: the order and the records first, the moment chain next, a real/Kelvin
  // launch beside the chain last, so that its CTAs take only what the chains leave free;
  // k_order_keys also zeroes both pair work counters (ctr_pairs_d and ctr_pairs2_d, adjacent),
  // which the pair launches use only after ev_img.  The items a launch takes statically (one
  // per worker, `first`) belong to the launch that has the list as its first list.
  const PairWork rk{it4x_d, L.nRK, ctr_pairs2_d, side_rk ? std::min(grid_rk * nw, L.nRK) : 0};
  const PairWork srf{it4x_d + L.nRK, nS, ctr_pairs_d, std::min(grid_s * nw, nS)}, none{nullptr, 0, nullptr, 0};
  {
    PriorityScope ps(prio_hi);
    launch_order(sys_d, nsys, itord_d, (int)L.itord.size(), itsort_d, (int)L.itsort.size(), indesc_d, xyz_d, q_d,
                 key_d, hist_d, sortscr_d, perm_d, xs_d, status_d, ctr_pairs_d, 2, L.order_smem_n, side);
    launch_images(sys_d, itord_d, (int)L.itord.size(), xyz_d, q_d, xs_d, perm_d, iperm_d, srchi_d, srclo_d, src64_d,
                  boxes_d, prec, status_d, side);
  }
  cudaEventRecord(ev_img, side);
  if (side_rk) {
    // a programmatic dependent of k_images (which does not trigger early): its launch is set up
    // while the records are written, and its CTAs start as soon as they are done
    launch_pair_items(rk, none, grid_rk, side, true);
    cudaEventRecord(ev_join, side);
  } else if (L.tree) {
    // the far-field tree (build and evaluation) beside the coefficient chain
    issue_tree(side);
    cudaEventRecord(ev_join, side);
  }
  PriorityScope ps(prio_mid);
  issue_moments();
  // the records are joined before the coefficients (done by then), so that the main stream's
  // pair launch has a single dependency and starts as a programmatic dependent of the surface
  cudaStreamWaitEvent(stream, ev_img, 0);
  launch_coef_reduce(sys_d, it2r_d, (int)L.it2r.size(), mom_d, L.mom_stride, Mn_d, coef_d, coef2_d, r0_d, prec,
                     stream);
  launch_surface(sys_d, L.use_sb ? it3m_d : it3_d, (int)(L.use_sb ? L.it3m.size() : L.it3.size()), L.maxP,
                 L.surf_pw, coef_d, coef2_d, sb_d, tables(), surfa_d, surfb_d, surf64a_d, surf64b_d, surfx_d,
                 surfqd_d, prec, stream);
  launch_pair_items(srf, rk, grid_s, stream, true);
  if (side_rk || L.tree) cudaStreamWaitEvent(stream, ev_join, 0);
  launch_reduce(sys_d, sel_d, selrng_d, nsys, it5_d, (int)L.it5.size(), part_d, part64_d, prec, q_d, perm_d, r0_d,
                phic_d, phir_d, phit_d, epart_d, nullptr, ctr_red_d, status_d, outdesc_d, stream, true);
}

// CTAs per SM of a real/Kelvin launch beside the coefficient chain.  Its persistent CTAs keep
// their SM's registers until the real/Kelvin items run out, so the chain's kernels run only in
// what it leaves free.  Schedule 1 leaves one CTA slot per SM (when there are at least four):
// 0.326 against 0.334 ms per step at N = 20000 with none left, 0.342 with two.  A slot of a
// small pair CTA may not hold a coefficient or surface CTA, which then waits for pair CTAs to
// finish (4 us per step for two cavities of N = 2000 with 64-thread pair CTAs); schedule 2
// leaves the registers of the largest of those CTAs instead.
int Engine::side_ctas_per_sm(int occ) const
{
  if (rk_side == 2 && prec != HSMA_FP64) {
    const int cta = std::max(regs_f32[L.cfg], 1);
    int per = occ;
    while (per > 1 && (int64_t)per * cta + chain_regs > sm_regs) --per;
    return per;
  }
  return occ >= 4 ? occ - 1 : occ;
}

int Engine::fused_launch_count() const
{
  if (L.itord.empty()) return build_launch_count() + pot_launch_count();
  return build_launch_count() + (rk_side != 0 && L.nRK > 0 ? 1 : 0) + (L.it4x.empty() ? 0 : 1) +
         (L.it5.empty() ? 0 : 1) + (L.tree ? tree_launch_count() : 0);
}

int Engine::run_graph(cudaGraphExec_t* g, void (Engine::*issue)())
{
  if (!use_graphs) {
    (this->*issue)();
    CK(cudaGetLastError());
    return HSMA_OK;
  }
  if (!*g) {
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
    (this->*issue)();
    cudaError_t e = cudaStreamEndCapture(stream, &graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(g, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      *g = nullptr;
      return cuda_fail(e, "cudaGraphInstantiate");
    }
  }
  CK(cudaGraphLaunch(*g, stream));
  return HSMA_OK;
}

// The device address of page-locked host memory (registered or allocated through CUDA), else
// null (pageable memory, or not host memory).
const void* pinned_device_address(const void* p)
{
  cudaPointerAttributes a{};
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// Pageable host inputs are copied to xyz_d, q_d now.  Device inputs and page-locked host inputs
// are not copied: the build pass (run by the next evaluation) reads them in place through the
// inputs descriptor, and its first kernel writes the engine's own copy, so such a step has no
// copy launches.
int Engine::build(const double* xyz, const double* q, bool device_inputs)
{
  CK(cudaSetDevice(device));
  const int64_t n = L.totN;
  in_pending = false;
  const double *xyz_in = device_inputs ? xyz : nullptr, *q_in = device_inputs ? q : nullptr;
  if (n > 0 && !device_inputs) {
    xyz_in = static_cast<const double*>(pinned_device_address(xyz));
    q_in = static_cast<const double*>(pinned_device_address(q));
  }
  if (n > 0 && xyz_in && q_in) {
    in_user = InDesc{xyz_in, q_in, 1, 0};
    in_pending = true;
  } else if (n > 0) {
    enter();
    CK(cudaMemcpyAsync(xyz_d, xyz, 24 * n, cudaMemcpyHostToDevice, stream));
    CK(cudaMemcpyAsync(q_d, q, 8 * n, cudaMemcpyHostToDevice, stream));
    leave();
  }
  sources_ready = true;
  build_pending = true;
  pot_ready = false;
  v_ready = false;
  return HSMA_OK;
}

// The inputs descriptor for a build pass about to be launched: the pending device inputs, else
// the engine's own arrays (a copy of the descriptor only when it changes: none per step when the
// caller builds from the same device arrays every step, or always from host arrays).
int Engine::prepare_inputs()
{
  const InDesc want = in_pending ? in_user : InDesc{xyz_d, q_d, 0, 0};
  if (!in_loaded || want.xyz != in_cur.xyz || want.q != in_cur.q || want.copy != in_cur.copy) {
    in_cur = want;
    CK(cudaMemcpyAsync(indesc_d, &in_cur, sizeof(InDesc), cudaMemcpyHostToDevice, stream));
    in_loaded = true;
  }
  in_pending = false;
  return HSMA_OK;
}

int Engine::ensure_built()
{
  if (!build_pending) return HSMA_OK;
  CK(cudaSetDevice(device));
  enter();
  int rc = prepare_inputs();
  if (rc) return rc;
  rc = run_graph(&g_build, &Engine::issue_build);
  if (rc) return rc;
  leave();
  launches += build_launch_count();
  build_pending = false;
  return HSMA_OK;
}

// Destinations of the next potential pass (OutDesc): rewritten on the device only when they
// change (a pageable source: the copy has taken it when the call returns).
int Engine::set_outputs(const OutDesc& od)
{
  if (od.phi == out_cur.phi && od.epart == out_cur.epart && od.status == out_cur.status && od.what == out_cur.what)
    return HSMA_OK;
  out_cur = od;
  CK(cudaMemcpyAsync(outdesc_d, &out_cur, sizeof(OutDesc), cudaMemcpyHostToDevice, stream));
  return HSMA_OK;
}

int Engine::potentials(const OutDesc& od, bool* wrote)
{
  if (wrote) *wrote = false;
  if (!sources_ready) return fail(HSMA_E_STATE, "sources have not been built");
  if (pot_ready) return HSMA_OK;
  CK(cudaSetDevice(device));
  {
    const int rs = set_outputs(od);
    if (rs) return rs;
  }
  if (build_pending && overlap) {
    enter();
    int rc = prepare_inputs();
    if (rc) return rc;
    rc = run_graph(&g_fused, &Engine::issue_fused);
    if (rc) return rc;
    leave();
    launches += fused_launch_count();
    build_pending = false;
  } else {
    int rc = ensure_built();
    if (rc) return rc;
    enter();
    rc = run_graph(&g_pot, &Engine::issue_pot);
    if (rc) return rc;
    leave();
    launches += pot_launch_count();
    if (!L.it4.empty()) pair_timed = true;
  }
  pot_ready = true;
  ++pot_epoch;
  energy_parts = true;  // the potential passes leave the energies as per-block terms (epart)
  field_ready = false;
  if (wrote) *wrote = true;
  return HSMA_OK;
}

// Enqueue the copy of every system's energies to the pinned mirror (after a potential pass on the
// engine's stream); valid once the stream has been synchronised.
int Engine::stage_energies()
{
  const size_t bytes = energy_parts ? 16 * L.it5.size() : 16 * L.sd.size();
  if (bytes > energy_h_cap) return fail(HSMA_E_STATE, "energy staging buffer not allocated");
  if (bytes)
    CK(cudaMemcpyAsync(energy_h, energy_parts ? epart_d : energy_d, bytes, cudaMemcpyDeviceToHost, stream));
  energy_h_parts = energy_parts;
  return HSMA_OK;
}

// Every system's (E_total, E_rf) from the raw energies of a pass: the per-block terms of the
// potential passes summed per system in block order, or the device-completed pairs.
void Engine::energies_from(const double* raw, bool parts, double* out) const
{
  for (size_t s = 0; s < L.sd.size(); ++s) {
    if (!parts) {
      out[2 * s] = raw[2 * s];
      out[2 * s + 1] = raw[2 * s + 1];
      continue;
    }
    double a = 0.0, b = 0.0;
    const int b0 = L.sd[s].k5_first, nb = L.sd[s].k5_count;
    for (int k = 0; k < nb; ++k) {
      a += raw[2 * (b0 + k)];
      b += raw[2 * (b0 + k) + 1];
    }
    out[2 * s] = a;
    out[2 * s + 1] = b;
  }
}

// Energies of the current potentials into out (2 per system), with the status check.
// Energies of the current pass through the pinned mirror (one round trip with the status);
// later reads of the same pass take the mirror without a copy.
int Engine::read_energies(double* out)
{
  if (!(energy_h && energy_h_epoch == pot_epoch)) {
    int rc = ensure_host_stage(0);
    if (rc) return rc;
    rc = stage_energies();
    if (rc) return rc;
    rc = check_status();
    if (rc) return rc;
    energy_h_epoch = pot_epoch;
  }
  energies_from(energy_h, energy_h_parts, out);
  return HSMA_OK;
}

// The pinned staging buffers of copy_to_host and stage_energies; allocated before the call
// enqueues any work (an allocation is no place between an enqueued copy and its wait).
int Engine::ensure_host_stage(int64_t count)
{
  const size_t need_e = 16 * std::max<size_t>(std::max(L.sd.size(), L.it5.size()), 1);
  if (need_e > energy_h_cap) {
    if (energy_h) cudaFreeHost(energy_h);
    energy_h = nullptr;
    energy_h_cap = 0;
    CK(cudaHostAlloc((void**)&energy_h, need_e, cudaHostAllocMapped));
    energy_h_cap = need_e;
    CK(cudaHostGetDevicePointer((void**)&energy_h_dev, energy_h, 0));
  }
  const size_t need = 8 * (size_t)std::max<int64_t>(count, 0) + 256;
  if (need > host_stage_cap) {
    if (host_stage) cudaFreeHost(host_stage);
    host_stage = nullptr;
    host_stage_cap = 0;
    CK(cudaHostAlloc((void**)&host_stage, need, cudaHostAllocMapped));
    host_stage_cap = need;
    CK(cudaHostGetDevicePointer((void**)&host_stage_dev, host_stage, 0));
  }
  return HSMA_OK;
}

int Engine::ensure_field_buffers()
{
  const size_t need_p = std::max<size_t>(32 * (size_t)L.totPart, 256);
  const size_t need_e = std::max<size_t>(72 * (size_t)L.totN, 256);
  if (need_p <= fpart_cap && need_e <= E_cap) {
    Ec_d = E_d;
    Er_d = E_d + 3 * L.totN;
    Et_d = E_d + 6 * L.totN;
    return HSMA_OK;
  }
  CK(cudaStreamSynchronize(stream));
  if (g_field) cudaGraphExecDestroy(g_field);
  if (g_field_fused) cudaGraphExecDestroy(g_field_fused);
  g_field = g_field_fused = nullptr;
  if (need_p > fpart_cap) {
    if (fpart_d) cudaFree(fpart_d);
    fpart_d = nullptr;
    fpart_cap = 0;
    cudaError_t e = cudaMalloc(&fpart_d, need_p);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fpart_d = nullptr;
      return fail(HSMA_E_OOM, "cudaMalloc(%zu) for the field partials failed", need_p);
    }
    fpart_cap = need_p;
  }
  if (need_e > E_cap) {
    if (E_d) cudaFree(E_d);
    E_d = nullptr;
    E_cap = 0;
    cudaError_t e = cudaMalloc((void**)&E_d, need_e);
    if (e != cudaSuccess) {
      cudaGetLastError();
      E_d = nullptr;
      return fail(HSMA_E_OOM, "cudaMalloc(%zu) for the fields failed", need_e);
    }
    E_cap = need_e;
  }
  Ec_d = E_d;
  Er_d = E_d + 3 * L.totN;
  Et_d = E_d + 6 * L.totN;
  return HSMA_OK;
}

int Engine::field_slots() const
{
  return num_sms * std::max(prec == HSMA_FP64 ? occ_field64 : occ_field[L.cfg], 1);
}

void Engine::launch_field_items(PairWork w1, PairWork w2, int grid, cudaStream_t st, bool pdl)
{
  if (w1.nitems <= 0 && w2.nitems <= 0) return;
  if (prec == HSMA_FP64)
    launch_field_f64(grid, sys_d, w1, w2, src64_d, surf64a_d, surf64b_d, (dbl4*)fpart_d, st, pdl);
  else
    launch_field_f32(L.cfg, grid, sys_d, w1, w2, srchi_d, srclo_d, surfa_d, surfb_d, boxes_d, (float4*)fpart_d, st,
                     pdl);
}

void Engine::launch_field_reduce(cudaStream_t st)
{
  launch_reduce_field(sys_d, sel_d, selrng_d, (int)L.sd.size(), it5_d, (int)L.it5.size(), (const float4*)fpart_d,
                      (const dbl4*)fpart_d, prec, q_d, perm_d, r0_d, phic_d, phir_d, phit_d, Ec_d, Er_d, Et_d,
                      epart_d, energy_d, ctr_red_d, status_d, st);
}

void Engine::issue_field()
{
  cudaMemsetAsync(ctr_pairs_d, 0, sizeof(unsigned int), stream);
  if (!L.it4f.empty()) {
    cudaEventRecordWithFlags(ev_pair0, stream, cudaEventRecordExternal);
    const int nit = (int)L.it4f.size();
    const int grid = std::max(1, std::min(nit, field_slots()));
    const PairWork all{it4f_d, nit, ctr_pairs_d, std::min(grid, nit)}, none{nullptr, 0, nullptr, 0};
    launch_field_items(all, none, grid, stream);
    cudaEventRecordWithFlags(ev_pair1, stream, cudaEventRecordExternal);
  }
  launch_field_reduce(stream);
}

// Build and field pass in one graph, as issue_fused does for the potentials (the same
// schedule of the real/Kelvin field items: beside the moment chain or after it).
void Engine::issue_field_fused()
{
  const int nsys = (int)L.sd.size();
  const int nS = (int)L.it4fx.size() - L.nRKf;
  const int slots = field_slots();
  const bool side_rk = rk_side != 0 && L.nRKf > 0;
  const int grid_rk = std::max(1, std::min(L.nRKf, slots));
  const int grid_s = std::max(1, std::min(nS + L.nRKf, slots));
  cudaEventRecord(ev_fork, stream);
  cudaStreamWaitEvent(side, ev_fork, 0);
  const PairWork rk{it4fx_d, L.nRKf, ctr_pairs2_d, side_rk ? std::min(grid_rk, L.nRKf) : 0};
  const PairWork srf{it4fx_d + L.nRKf, nS, ctr_pairs_d, std::min(grid_s, nS)}, none{nullptr, 0, nullptr, 0};
  {
    PriorityScope ps(prio_hi);
    launch_order(sys_d, nsys, itord_d, (int)L.itord.size(), itsort_d, (int)L.itsort.size(), indesc_d, xyz_d, q_d,
                 key_d, hist_d, sortscr_d, perm_d, xs_d, status_d, ctr_pairs_d, 2, L.order_smem_n, side);
    launch_images(sys_d, itord_d, (int)L.itord.size(), xyz_d, q_d, xs_d, perm_d, iperm_d, srchi_d, srclo_d, src64_d,
                  boxes_d, prec, status_d, side);
  }
  cudaEventRecord(ev_img, side);
  if (side_rk) {
    launch_field_items(rk, none, grid_rk, side);
    cudaEventRecord(ev_join, side);
  }
  PriorityScope ps(prio_mid);
  issue_moments();
  cudaStreamWaitEvent(stream, ev_img, 0);  // (as in issue_fused)
  launch_coef_reduce(sys_d, it2r_d, (int)L.it2r.size(), mom_d, L.mom_stride, Mn_d, coef_d, coef2_d, r0_d, prec,
                     stream);
  launch_surface(sys_d, L.use_sb ? it3m_d : it3_d, (int)(L.use_sb ? L.it3m.size() : L.it3.size()), L.maxP,
                 L.surf_pw, coef_d, coef2_d, sb_d, tables(), surfa_d, surfb_d, surf64a_d, surf64b_d, surfx_d,
                 surfqd_d, prec, stream);
  launch_field_items(srf, rk, grid_s, stream, true);
  if (side_rk) cudaStreamWaitEvent(stream, ev_join, 0);
  launch_field_reduce(stream);
}

int Engine::field()
{
  if (L.tree && have_layout) return fail(HSMA_E_STATE, "fields are not available with the far-field tree");
  if (!sources_ready) return fail(HSMA_E_STATE, "sources have not been built");
  if (pot_ready && field_ready) return HSMA_OK;
  CK(cudaSetDevice(device));
  int rc = ensure_field_buffers();
  if (rc) return rc;
  if (build_pending && overlap && !L.itord.empty()) {
    enter();
    rc = prepare_inputs();
    if (rc) return rc;
    rc = run_graph(&g_field_fused, &Engine::issue_field_fused);
    if (rc) return rc;
    leave();
    launches += build_launch_count() + (rk_side != 0 && L.nRKf > 0 ? 1 : 0) + (L.it4fx.empty() ? 0 : 1) +
                (L.it5.empty() ? 0 : 1);
    build_pending = false;
  } else {
    rc = ensure_built();
    if (rc) return rc;
    enter();
    rc = run_graph(&g_field, &Engine::issue_field);
    if (rc) return rc;
    leave();
    launches += pot_launch_count();
    if (!L.it4.empty()) pair_timed = true;
  }
  pot_ready = true;
  ++pot_epoch;
  energy_parts = false;  // the field pass completes the energies on the device
  field_ready = true;
  return HSMA_OK;
}

int Engine::check_status()
{
  // the status word through pinned memory (a pageable copy costs a driver-staged round trip)
  int rc = ensure_host_stage(0);
  if (rc) return rc;
  int* st_h = reinterpret_cast<int*>(host_stage);
  CK(cudaMemcpyAsync(st_h, status_d, sizeof(int), cudaMemcpyDeviceToHost, stream));
  CK(cudaStreamSynchronize(stream));
  return decode_status(*st_h);
}

// Copy count doubles from the device to caller host memory through a pinned staging buffer,
// with the energies (pinned mirror) and the status word in the same round trip, then decode the
// status: one stream synchronisation instead of one per pageable copy.
int Engine::out_lane(int what) { return what == HSMA_COULOMB ? 0 : (what == HSMA_REACTION ? 1 : 2); }

// Pinned staging of a host-output pass: values at byte 256, the status bytes at byte 16 (zeroed
// here: the staging buffer is written only by passes that a host-output call waits for).
// phi_dev: the device address of the caller's page-locked output array (written there directly),
// else null (written to the staging buffer and copied out by copy_to_host)
OutDesc Engine::host_outputs(int64_t count, int what, double* phi_dev)
{
  std::memset(host_stage + 16, 0, kStBits);
  return OutDesc{count > 0 ? (phi_dev ? phi_dev : host_stage_dev + 32) : nullptr, energy_h_dev,
                 reinterpret_cast<unsigned char*>(host_stage_dev) + 16, out_lane(what), 0};
}

int Engine::copy_to_host(const double* src_d, int64_t count, double* dst_h, bool written, bool direct)
{
  if (8 * (size_t)std::max<int64_t>(count, 0) + 256 > host_stage_cap)
    return fail(HSMA_E_STATE, "host staging buffer not allocated");
  int* st_h = reinterpret_cast<int*>(host_stage);
  double* vals = reinterpret_cast<double*>(host_stage + 256);
  int st = 0;
  if (written) {
    // the pass wrote the values, its per-block energy terms and its status bytes
    energy_h_parts = true;
    CK(cudaStreamSynchronize(stream));
    const unsigned char* sb = reinterpret_cast<const unsigned char*>(host_stage) + 16;
    for (int b = 0; b < kStBits; ++b)
      if (sb[b]) st |= 1 << b;
  } else {
    if (count > 0)
      CK(cudaMemcpyAsync(direct ? dst_h : vals, src_d, 8 * (size_t)count, cudaMemcpyDeviceToHost, stream));
    const int rs = stage_energies();
    if (rs) return rs;
    CK(cudaMemcpyAsync(st_h, status_d, sizeof(int), cudaMemcpyDeviceToHost, stream));
    CK(cudaStreamSynchronize(stream));
    st = *st_h;
  }
  const int rc = decode_status(st);
  if (rc) return rc;
  if (count > 0 && !direct) std::memcpy(dst_h, vals, 8 * (size_t)count);
  energy_h_epoch = pot_epoch;
  return HSMA_OK;
}

int Engine::decode_status(int st)
{
  if (st) {
    CK(cudaMemsetAsync(status_d, 0, sizeof(int), stream));
    pot_ready = false;
    if (st & kStOutside) {
      sources_ready = false;
      return fail(HSMA_E_OUTSIDE, "a charge lies outside the cavity (|x| >= a) or is not finite");
    }
    if (st & kStBadMove) return fail(HSMA_E_OUTSIDE, "moved charge outside the cavity");
    if (st & kStNonFinite)
      return fail(HSMA_E_NONFINITE, "non-finite potential (coincident charges?)");
  }
  return HSMA_OK;
}

// Pair-sum tile configuration for a set of sizes: the autotuned choice if one is cached for
// this size bucket, else a size heuristic.
int Engine::choose_config(const std::vector<int64_t>& ns) const
{
  if (forced_cfg >= 0) return forced_cfg;
  int64_t tot = 0;
  for (auto v : ns) tot += v;
  const int bucket = tune_bucket(tot, (int)ns.size());
  for (const auto& e : tuned)
    if (e.bucket == bucket) return e.cfg;
  return 0;
}

// Schedule of the real/Kelvin pair items in the fused graph: forced, else the size class's
// tuned choice, else beside the moment chain for a few cavities and after it for many (the
// faster one on the single-cavity and two-cavity workloads and on a batch of 512 measured).
int Engine::choose_side(const std::vector<int64_t>& ns) const
{
  if (forced_side >= 0) return forced_side;
  int64_t tot = 0;
  for (auto v : ns) tot += v;
  const int bucket = tune_bucket(tot, (int)ns.size());
  for (const auto& e : tuned)
    if (e.bucket == bucket) return e.side;
  return ns.size() <= 8 ? 1 : 0;
}

int tune_bucket(int64_t total_n, int nsys)
{
  int b = 0;
  int64_t v = std::max<int64_t>(total_n, 1);
  while (v > 1) {
    v >>= 1;
    ++b;
  }
  return b * 2 + (nsys > 1 ? 1 : 0);
}

}  // namespace hsma

// =======================================================================================
// C ABI
// =======================================================================================
using hsma::Engine;

struct hsma_t {
  Engine* e = nullptr;
  int64_t n = -1;
  std::string err;
};

static int validate_params(const hsma_params* p, std::string& why)
{
  if (!p) {
    why = "params is NULL";
    return HSMA_E_INVALID_ARG;
  }
  if (p->p < 0 || p->p > HSMA_P_MAX) {
    why = "p out of range [0, HSMA_P_MAX]";
    return HSMA_E_INVALID_ARG;
  }
  if (p->F2 > 0) {
    if (p->F1 <= 0 || p->F1 >= p->F2) {
      why = "need 0 < F1 < F2";
      return HSMA_E_INVALID_ARG;
    }
  } else if (p->M < 4 || (p->M % 2) != 0) {
    why = "M must be even and >= 4";
    return HSMA_E_INVALID_ARG;
  }
  if (!(p->tau > 0.0) || !std::isfinite(p->tau)) {
    why = "tau must be > 0";
    return HSMA_E_INVALID_ARG;
  }
  if (!(p->dy_rel > 0.0) || !(p->dy_rel < 0.5) || !std::isfinite(p->dy_rel)) {
    why = "dy_rel must be in (0, 0.5)";
    return HSMA_E_INVALID_ARG;
  }
  if (!std::isfinite(p->coulomb_k)) {
    why = "coulomb_k must be finite";
    return HSMA_E_INVALID_ARG;
  }
  if (p->precision != HSMA_FP32 && p->precision != HSMA_FP64) {
    why = "precision must be HSMA_FP32 or HSMA_FP64";
    return HSMA_E_INVALID_ARG;
  }
  return HSMA_OK;
}

namespace hsma {
int make_spec(double a, double eps1, double eps2, double kappa, const hsma_params* prm, SysSpec* out, std::string& why)
{
  int rc = validate_params(prm, why);
  if (rc) return rc;
  if (!(a > 0.0) || !std::isfinite(a) || !(eps1 > 0.0) || !std::isfinite(eps1) || !(eps2 > 0.0) ||
      !std::isfinite(eps2) || !(kappa >= 0.0) || !std::isfinite(kappa)) {
    why = "need a > 0, eps1 > 0, eps2 > 0, kappa >= 0 (finite)";
    return HSMA_E_INVALID_ARG;
  }
  SysSpec s;
  s.a = a;
  s.eps1 = eps1;
  s.eps2 = eps2;
  s.kappa = kappa;
  s.tau = prm->tau;
  s.dy_rel = prm->dy_rel;
  s.coulk = prm->coulomb_k;
  s.p = prm->p;
  if (prm->F2 > 0) {
    s.F2 = prm->F2;
    s.F1 = prm->F1;
  } else {
    s.F2 = prm->M / 2 - 1;
    s.F1 = (int)std::lround(s.F2 * (std::sqrt(5.0) - 1.0) / 2.0);
  }
  s.M = 2 * (s.F2 + 1);
  *out = s;
  return HSMA_OK;
}
}  // namespace hsma

static int set_err(hsma_t* h, int code, const char* msg)
{
  if (h) h->err = msg;
  return code;
}

static int from_engine(hsma_t* h, int rc)
{
  if (rc != HSMA_OK) h->err = h->e->err;
  return rc;
}

extern "C" {

const char* hsma_version(void) { return "hsma-gb300 0.1 (sm_103a)"; }

int hsma_default_params(hsma_params* p)
{
  if (!p) return HSMA_E_INVALID_ARG;
  memset(p, 0, sizeof(*p));
  p->p = 20;
  p->M = 1000;
  p->F1 = 0;
  p->F2 = 0;
  p->tau = 0.1;
  p->dy_rel = 1e-5;
  p->coulomb_k = 1.0 / (4.0 * hsma::kPi);
  p->precision = HSMA_FP32;
  p->device = 0;
  p->stream = nullptr;
  return HSMA_OK;
}

int hsma_create(double a, double eps1, double eps2, double kappa, const hsma_params* params, hsma_t** out)
{
  if (!out) return HSMA_E_INVALID_ARG;
  *out = nullptr;
  std::string why;
  hsma::SysSpec s;
  int rc = hsma::make_spec(a, eps1, eps2, kappa, params, &s, why);
  if (rc) return rc;
  hsma_t* h = new hsma_t();
  h->e = new Engine();
  h->e->spec.push_back(s);
  rc = h->e->init(params->device, params->stream, params->precision);
  if (rc) {
    delete h->e;
    delete h;
    return rc;
  }
  *out = h;
  return HSMA_OK;
}

void hsma_destroy(hsma_t* h)
{
  if (!h) return;
  delete h->e;
  delete h;
}

const char* hsma_last_error(const hsma_t* h)
{
  if (!h) return "NULL handle";
  return h->err.c_str();
}

int hsma_workspace_size(hsma_t* h, int64_t n, size_t* bytes)
{
  if (!h || !bytes || n < 0 || n > (int64_t)INT32_MAX / 4) return set_err(h, HSMA_E_INVALID_ARG, "bad argument");
  const int cfg = h->e->prec == HSMA_FP64 ? 0 : h->e->choose_config({n});
  *bytes = h->e->make_layout({n}, cfg).bytes;
  return HSMA_OK;
}

int hsma_attach_workspace(hsma_t* h, void* device_ptr, size_t bytes)
{
  if (!h) return HSMA_E_INVALID_ARG;
  h->n = -1;
  return from_engine(h, h->e->attach(device_ptr, bytes));
}

static int build_common(hsma_t* h, int64_t n, const double* xyz, const double* q, bool dev)
{
  if (!h) return HSMA_E_INVALID_ARG;
  if (n < 0 || n > (int64_t)INT32_MAX / 4) return set_err(h, HSMA_E_INVALID_ARG, "n out of range");
  if (n > 0 && (!xyz || !q)) return set_err(h, HSMA_E_INVALID_ARG, "NULL xyz or q");
  // (every charge is checked by the pass's first kernel, k_order_keys, for host and device
  // inputs alike: the evaluation that runs the pass returns HSMA_E_OUTSIDE)
  int rc = h->e->set_sizes({n});
  if (rc) return from_engine(h, rc);
  h->n = n;
  return from_engine(h, h->e->build(xyz, q, dev));
}

int hsma_build_sources(hsma_t* h, int64_t n, const double* xyz, const double* q)
{
  return build_common(h, n, xyz, q, false);
}

int hsma_build_sources_device(hsma_t* h, int64_t n, const double* xyz_dev, const double* q_dev)
{
  return build_common(h, n, xyz_dev, q_dev, true);
}

static const double* pick_phi(Engine* e, int what)
{
  if (what == HSMA_TOTAL) return e->phit_d;
  if (what == HSMA_REACTION) return e->phir_d;
  if (what == HSMA_COULOMB) return e->phic_d;
  return nullptr;
}

int hsma_potential(hsma_t* h, double* phi, int what)
{
  if (!h) return HSMA_E_INVALID_ARG;
  if (h->n < 0) return set_err(h, HSMA_E_STATE, "sources have not been built");
  if (h->n > 0 && !phi) return set_err(h, HSMA_E_INVALID_ARG, "NULL phi");
  const double* src = pick_phi(h->e, what);
  if (!src) return set_err(h, HSMA_E_INVALID_ARG, "bad 'what'");
  int rc = h->e->ensure_host_stage(h->n);
  if (rc) return from_engine(h, rc);
  bool wrote = false;
  double* phi_dev = static_cast<double*>(const_cast<void*>(hsma::pinned_device_address(phi)));
  rc = h->e->potentials(h->e->host_outputs(h->n, what, phi_dev), &wrote);
  if (rc) return from_engine(h, rc);
  return from_engine(h, h->e->copy_to_host(src, h->n, phi, wrote, phi_dev != nullptr));
}

int hsma_potential_device(hsma_t* h, double* phi_dev, int what)
{
  if (!h) return HSMA_E_INVALID_ARG;
  if (h->n < 0) return set_err(h, HSMA_E_STATE, "sources have not been built");
  if (h->n > 0 && !phi_dev) return set_err(h, HSMA_E_INVALID_ARG, "NULL phi");
  const double* src = pick_phi(h->e, what);
  if (!src) return set_err(h, HSMA_E_INVALID_ARG, "bad 'what'");
  bool wrote = false;
  const hsma::OutDesc od{h->n > 0 ? phi_dev : nullptr, nullptr, nullptr, Engine::out_lane(what), 0};
  int rc = h->e->potentials(od, &wrote);
  if (rc) return from_engine(h, rc);
  if (h->n > 0 && !wrote) {
    cudaError_t e = cudaMemcpyAsync(phi_dev, src, 8 * h->n, cudaMemcpyDeviceToDevice, h->e->stream);
    if (e != cudaSuccess) return from_engine(h, h->e->cuda_fail(e, "copy phi"));
  }
  return HSMA_OK;
}

static const double* pick_field(Engine* e, int what)
{
  if (what == HSMA_TOTAL) return e->Et_d;
  if (what == HSMA_REACTION) return e->Er_d;
  if (what == HSMA_COULOMB) return e->Ec_d;
  return nullptr;
}

static int field_out(hsma_t* h, double* E, int what, bool dev)
{
  if (!h) return HSMA_E_INVALID_ARG;
  if (h->n < 0) return set_err(h, HSMA_E_STATE, "sources have not been built");
  if (h->n > 0 && !E) return set_err(h, HSMA_E_INVALID_ARG, "NULL E");
  if (what != HSMA_TOTAL && what != HSMA_REACTION && what != HSMA_COULOMB)
    return set_err(h, HSMA_E_INVALID_ARG, "bad 'what'");
  int rc = dev ? HSMA_OK : h->e->ensure_host_stage(3 * h->n);
  if (rc) return from_engine(h, rc);
  rc = h->e->field();
  if (rc) return from_engine(h, rc);
  if (!dev) return from_engine(h, h->e->copy_to_host(pick_field(h->e, what), 3 * h->n, E));
  if (h->n > 0) {
    cudaError_t e = cudaMemcpyAsync(E, pick_field(h->e, what), 24 * h->n, cudaMemcpyDeviceToDevice, h->e->stream);
    if (e != cudaSuccess) return from_engine(h, h->e->cuda_fail(e, "copy E"));
  }
  return HSMA_OK;
}

int hsma_field(hsma_t* h, double* E, int what) { return field_out(h, E, what, false); }
int hsma_field_device(hsma_t* h, double* E_dev, int what) { return field_out(h, E_dev, what, true); }

int hsma_energy(hsma_t* h, double* e_total, double* e_reaction)
{
  if (!h) return HSMA_E_INVALID_ARG;
  if (h->n < 0) return set_err(h, HSMA_E_STATE, "sources have not been built");
  int rc = h->e->potentials();
  if (rc) return from_engine(h, rc);
  double en[2] = {0.0, 0.0};
  rc = h->e->read_energies(en);
  if (rc) return from_engine(h, rc);
  if (e_total) *e_total = en[0];
  if (e_reaction) *e_reaction = en[1];
  return HSMA_OK;
}

int hsma_delta_energy(hsma_t* h, int64_t k, const double* x_new, double* de)
{
  if (!h) return HSMA_E_INVALID_ARG;
  return from_engine(h, h->e->delta_energy(k, x_new, de));
}

int hsma_apply_move(hsma_t* h, int64_t k, const double* x_new)
{
  if (!h) return HSMA_E_INVALID_ARG;
  return from_engine(h, h->e->apply_move(k, x_new));
}

int hsma_set_overlap(hsma_t* h, int on)
{
  if (!h) return HSMA_E_INVALID_ARG;
  h->e->overlap = on != 0;
  return HSMA_OK;
}

int64_t hsma_kernel_launches(const hsma_t* h) { return h ? h->e->launches : 0; }

int hsma_coefficients(hsma_t* h, double* out, int64_t len)
{
  if (!h || !out) return HSMA_E_INVALID_ARG;
  if (h->n < 0 || !h->e->sources_ready) return set_err(h, HSMA_E_STATE, "sources have not been built");
  const int P = h->e->L.sd[0].P;
  if (len < P) return set_err(h, HSMA_E_INVALID_ARG, "output shorter than (p+1)^2");
  int rc = h->e->ensure_built();
  if (rc) return from_engine(h, rc);
  cudaError_t e = cudaMemcpyAsync(out, h->e->coef_d, 8 * (size_t)P, cudaMemcpyDeviceToHost, h->e->stream);
  if (e != cudaSuccess) return from_engine(h, h->e->cuda_fail(e, "copy coefficients"));
  return from_engine(h, h->e->check_status());
}

int hsma_last_pair_time(hsma_t* h, float* ms)
{
  if (!h || !ms) return HSMA_E_INVALID_ARG;
  return from_engine(h, h->e->last_pair_time(ms));
}

int hsma_set_far_field(hsma_t* h, double theta, int order)
{
  if (!h) return HSMA_E_INVALID_ARG;
  if (!(theta == 0.0 || (theta > 0.0 && theta < 1.0)))
    return set_err(h, HSMA_E_INVALID_ARG, "theta must be 0 (direct sum) or in (0, 1)");
  if (theta > 0.0 && !hsma::tree_order_supported(order))
    return set_err(h, HSMA_E_INVALID_ARG, "far-field order must be 8, 12 or 16");
  if (theta > 0.0 && h->e->prec != HSMA_FP32)
    return set_err(h, HSMA_E_INVALID_ARG, "the far-field tree needs the FP32 path");
  h->e->far_theta = theta;
  if (theta > 0.0) h->e->far_order = order;
  // a new layout and a new build pass at the next call
  h->e->layout_uploaded = false;
  h->e->sources_ready = false;
  h->e->build_pending = false;
  h->n = -1;
  return HSMA_OK;
}

int hsma_last_far_time(hsma_t* h, float* ms)
{
  if (!h || !ms) return HSMA_E_INVALID_ARG;
  return from_engine(h, h->e->last_tree_time(ms));
}

}  // extern "C"

namespace hsma {

// Potentials of the real charges under the surface kernels (needed by Delta E); computed once
// per build and then updated by committed moves.
int Engine::ensure_v()
{
  if (v_ready) return HSMA_OK;
  if (!L.it3.empty()) {
    launch_surface_potentials(sys_d, it3_d, (int)L.it3.size(), xyz_d, q_d, surfx_d, vsurf_d, stream);
    CK(cudaGetLastError());
    launches += 1;
  }
  v_ready = true;
  return HSMA_OK;
}

static int check_moves(Engine& e, const std::vector<DeltaReq>& reqs)
{
  if ((int)reqs.size() > e.L.max_req)
    return e.fail(HSMA_E_INVALID_ARG, "%zu move requests exceed the reserved %d", reqs.size(), e.L.max_req);
  for (const auto& r : reqs) {
    if (r.sys < 0 || r.sys >= (int)e.L.sd.size()) return e.fail(HSMA_E_INVALID_ARG, "bad system index");
    const SysDev& d = e.L.sd[r.sys];
    if (r.k < 0 || r.k >= d.n) return e.fail(HSMA_E_INVALID_ARG, "charge index %d out of range", r.k);
    const double r2 = r.x * r.x + r.y * r.y + r.z * r.z;
    if (!(r2 < d.a * d.a) || !std::isfinite(r2)) return e.fail(HSMA_E_OUTSIDE, "moved charge outside the cavity");
  }
  return HSMA_OK;
}

int Engine::delta_batch(const std::vector<DeltaReq>& reqs, double* de_host)
{
  if (!sources_ready) return fail(HSMA_E_STATE, "sources have not been built");
  int rc = check_moves(*this, reqs);
  if (rc) return rc;
  rc = ensure_built();
  if (rc) return rc;
  if (reqs.empty()) return HSMA_OK;
  std::vector<int4> items;
  std::vector<int2> ranges(reqs.size());
  for (size_t r = 0; r < reqs.size(); ++r) {
    const SysDev& d = L.sd[reqs[r].sys];
    ranges[r].x = (int)items.size();
    for (int b = 0; b < (d.n + kDeltaBlock - 1) / kDeltaBlock; ++b) items.push_back(make_int4((int)r, 0, b, 0));
    for (int b = 0; b < (d.M + kDeltaBlock - 1) / kDeltaBlock; ++b) items.push_back(make_int4((int)r, 1, b, 0));
    ranges[r].y = (int)items.size() - ranges[r].x;
  }
  CK(cudaSetDevice(device));
  enter();
  rc = ensure_v();
  if (rc) return rc;
  CK(cudaMemcpyAsync(dreq_d, reqs.data(), sizeof(DeltaReq) * reqs.size(), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(ditems_d, items.data(), sizeof(int4) * items.size(), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(dreqit_d, ranges.data(), sizeof(int2) * ranges.size(), cudaMemcpyHostToDevice, stream));
  launch_delta(sys_d, ditems_d, (int)items.size(), dreqit_d, dreq_d, (int)reqs.size(), xyz_d, q_d, perm_d, iperm_d,
               srchi_d, srclo_d, src64_d, surfx_d, surfqd_d, vsurf_d, Mn_d, tables(), dpart_d, de_d, ctr_delta_d,
               status_d, stream);
  CK(cudaGetLastError());
  launches += 1;
  CK(cudaMemcpyAsync(de_host, de_d, 8 * reqs.size(), cudaMemcpyDeviceToHost, stream));
  leave();
  return check_status();
}

int Engine::move_batch(const std::vector<DeltaReq>& reqs)
{
  if (!sources_ready) return fail(HSMA_E_STATE, "sources have not been built");
  int rc = check_moves(*this, reqs);
  if (rc) return rc;
  rc = ensure_built();
  if (rc) return rc;
  if (reqs.empty()) return HSMA_OK;
  std::vector<int2> items;
  for (size_t r = 0; r < reqs.size(); ++r) {
    for (size_t o = 0; o < r; ++o)
      if (reqs[o].sys == reqs[r].sys) return fail(HSMA_E_INVALID_ARG, "two moves of one system in a batch");
    const SysDev& d = L.sd[reqs[r].sys];
    for (int b = 0; b < (d.M + kDeltaBlock - 1) / kDeltaBlock; ++b) items.push_back(make_int2((int)r, b));
  }
  CK(cudaSetDevice(device));
  enter();
  CK(cudaMemcpyAsync(dreq_d, reqs.data(), sizeof(DeltaReq) * reqs.size(), cudaMemcpyHostToDevice, stream));
  CK(cudaMemcpyAsync(mitems_d, items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice, stream));
  launch_move(sys_d, mitems_d, (int)items.size(), dreq_d, (int)reqs.size(), tables(), L.maxP, xyz_d, q_d, Mn_d,
              coef_d, coef2_d, r0_d, surfx_d, surfqd_d, vsurf_d, v_ready ? 1 : 0, surfa_d, surfb_d, surf64a_d,
              surf64b_d, iperm_d, srchi_d, srclo_d, src64_d, boxes_d, stream);
  CK(cudaGetLastError());
  leave();
  launches += items.empty() ? 1 : 2;
  pot_ready = false;
  return HSMA_OK;
}

int Engine::delta_energy(int64_t k, const double* x_new, double* de)
{
  if (L.tree && have_layout) return fail(HSMA_E_STATE, "single-move energies are not available with the far-field tree");
  if (!x_new || !de) return fail(HSMA_E_INVALID_ARG, "NULL argument");
  if (L.sd.empty()) return fail(HSMA_E_STATE, "sources have not been built");
  DeltaReq r;
  r.sys = 0;
  r.k = (int)std::min<int64_t>(std::max<int64_t>(k, -1), INT32_MAX);
  r.x = x_new[0];
  r.y = x_new[1];
  r.z = x_new[2];
  return delta_batch({r}, de);
}

int Engine::apply_move(int64_t k, const double* x_new)
{
  if (L.tree && have_layout) return fail(HSMA_E_STATE, "moves are not available with the far-field tree");
  if (!x_new) return fail(HSMA_E_INVALID_ARG, "NULL argument");
  if (L.sd.empty()) return fail(HSMA_E_STATE, "sources have not been built");
  DeltaReq r;
  r.sys = 0;
  r.k = (int)std::min<int64_t>(std::max<int64_t>(k, -1), INT32_MAX);
  r.x = x_new[0];
  r.y = x_new[1];
  r.z = x_new[2];
  return move_batch({r});
}

}  // namespace hsma
