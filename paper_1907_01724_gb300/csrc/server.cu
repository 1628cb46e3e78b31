// Serving loop (include/hsma.h, hsma_server_*): Monte Carlo chains resident on the device,
// continuous batching of single-charge-move energy changes, overlapped full energies.
//
// * Live boundary: hsma_server_start runs the request loop on a native thread of its own;
//   producers call hsma_server_submit from any thread while it runs (a bounded inbound queue),
//   consumers take answers with hsma_server_poll (a host-side deadline), and hsma_server_stop
//   drains or cancels what is left.  hsma_server_run replays a request array through the same
//   loop (submitting each request at its release time from the calling thread).
// * Residency and admission: one batched Engine holds every resident chain.  A request for a
//   chain that is not resident waits in its chain's queue; it is admitted as soon as its
//   chain's device footprint fits the budget once idle resident chains (no request queued or
//   in flight, least recently used first) are evicted; the resident set is then rebuilt, at a
//   point where no work is in flight, from the host copy of every chain's committed state.  A
//   chain whose footprint alone exceeds the budget is answered HSMA_E_BUSY.
// * Ordering: a chain has at most one request in flight; its released requests wait in a
//   FIFO, so its results follow its own order whatever the mix.
// * Move requests: all ready move requests of idle chains form one batched k_delta launch on
//   a high-priority stream, followed in the same stream by the commit (k_move_surface,
//   k_move_charge) of the accepted ones; one such batch is in flight at a time.
// * Energy requests: each runs on its own low-priority stream slot as a sequence of pair-kernel
//   launches over bounded chunks of that chain's items (grids capped at a fraction of the GPU),
//   then k_reduce; between the chunks the block scheduler hands the freed SMs to the
//   high-priority move batches, so a large chain's energy does not hold the GPU for its whole
//   duration.
// * Completion is seen with cudaEventQuery; no device-side waits are involved.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "engine.h"

using hsma::DeltaReq;
using hsma::Engine;
using hsma::SysSpec;

namespace {

double now_s()
{
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// Pair work of one energy-request launch: items are split into chunks of about this many pair
// evaluations (~50 us of the capped grid) and at least one item per CTA of the capped grid, so
// that move batches get SMs between the launches of a large chain.
constexpr double kEnergyChunkPairs = 1.5e8;

// A request released to the loop: the caller's request, its ticket and submission time.
struct Pending {
  hsma_request q;
  int64_t ticket;
  double t_sub;  // server clock
};

struct EnergySlot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  int4* items_d = nullptr;
  int2* it5_d = nullptr;
  int* sel_d = nullptr;
  int2* selrng_d = nullptr;
  double* epart_d = nullptr;
  unsigned int* ctr_d = nullptr;
  int4* items_h = nullptr;
  int2* it5_h = nullptr;
  int* sel_h = nullptr;
  int2* selrng_h = nullptr;
  double* energy_h = nullptr;
  int live = 0;  // a request is in flight on this slot
  Pending p;
  int chain = -1;
};

}  // namespace

struct hsma_server_t {
  Engine* e = nullptr;
  hsma_params prm;
  std::vector<SysSpec> specs;                  // every chain
  std::vector<std::vector<double>> pos, chg;   // committed host state of every chain
  std::vector<int64_t> n;
  std::vector<size_t> footprint;
  std::vector<int> sys_of;                      // chain -> engine system, or -1
  std::vector<int> chain_of;                    // engine system -> chain
  std::vector<char> closed;
  size_t budget = 0;
  int max_batch = 64, energy_slots = 4;
  double sm_frac = 0.75;
  cudaStream_t sA = nullptr;
  cudaEvent_t evA = nullptr;
  std::vector<EnergySlot> slots;
  int items_cap = 0, it5_cap = 0;
  DeltaReq *dreq_h = nullptr, *mreq_h = nullptr, *mreq_d = nullptr;
  int4* ditems_h = nullptr;
  int2 *dranges_h = nullptr, *mitems_h = nullptr, *mitems_d = nullptr;
  double* de_h = nullptr;
  int ditems_cap = 0, mitems_cap = 0;
  std::vector<std::vector<int4>> it4_of;
  std::vector<std::vector<int2>> it5_of;
  std::string err;
  bool loaded = false;
  // live loop
  std::thread th;
  std::mutex mu;                       // inbox, outbox, counters, flags and pos
  std::condition_variable cv_loop, cv_out;
  std::deque<Pending> inbox;
  std::deque<hsma_result> outbox;
  int queue_cap = 1 << 16;             // submitted but not yet answered requests
  int64_t next_ticket = 0, in_system = 0;
  bool running = false, stop_req = false, drain = true;
  int loop_rc = HSMA_OK;
  double t0 = 0.0;                     // server clock origin (hsma_server_start)
  std::vector<double> last_used;       // per chain, server clock (least recently used eviction)
  std::vector<double> pairs_of;        // per resident system: pair evaluations of its item list
};

static int serr(hsma_server_t* s, int code, const std::string& msg)
{
  if (s) s->err = msg;
  return code;
}

static int scuda(hsma_server_t* s, cudaError_t e, const char* what)
{
  cudaGetLastError();
  return serr(s, HSMA_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SCK(call)                                \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return scuda(s, e_, #call); \
  } while (0)

static void free_buffers(hsma_server_t* s)
{
  for (auto& sl : s->slots) {
    if (sl.st) cudaStreamDestroy(sl.st);
    if (sl.ev) cudaEventDestroy(sl.ev);
    cudaFree(sl.items_d);
    cudaFree(sl.it5_d);
    cudaFree(sl.sel_d);
    cudaFree(sl.selrng_d);
    cudaFree(sl.epart_d);
    cudaFree(sl.ctr_d);
    cudaFreeHost(sl.items_h);
    cudaFreeHost(sl.it5_h);
    cudaFreeHost(sl.sel_h);
    cudaFreeHost(sl.selrng_h);
    cudaFreeHost(sl.energy_h);
    sl = EnergySlot();
  }
  cudaFreeHost(s->dreq_h);
  cudaFreeHost(s->mreq_h);
  cudaFreeHost(s->ditems_h);
  cudaFreeHost(s->dranges_h);
  cudaFreeHost(s->mitems_h);
  cudaFreeHost(s->de_h);
  cudaFree(s->mreq_d);
  cudaFree(s->mitems_d);
  s->dreq_h = s->mreq_h = s->mreq_d = nullptr;
  s->ditems_h = nullptr;
  s->dranges_h = s->mitems_h = s->mitems_d = nullptr;
  s->de_h = nullptr;
}

// Build the resident set: the engine holds the admitted chains, built from host state.
static int rebuild(hsma_server_t* s)
{
  Engine* e = s->e;
  std::vector<int64_t> ns;
  std::vector<SysSpec> sp;
  std::vector<double> xyz, q;
  s->chain_of.clear();
  for (size_t c = 0; c < s->specs.size(); ++c) {
    if (s->sys_of[c] < 0) continue;
    s->sys_of[c] = (int)s->chain_of.size();
    s->chain_of.push_back((int)c);
    sp.push_back(s->specs[c]);
    ns.push_back(s->n[c]);
    xyz.insert(xyz.end(), s->pos[c].begin(), s->pos[c].end());
    q.insert(q.end(), s->chg[c].begin(), s->chg[c].end());
  }
  if (sp.empty()) return HSMA_OK;
  e->spec = sp;
  e->max_requests = s->max_batch;
  e->layout_uploaded = false;
  e->drop_graphs();
  int rc = e->set_sizes(ns);
  if (rc) return serr(s, rc, e->err);
  rc = e->build(xyz.data(), q.data(), false);
  if (rc) return serr(s, rc, e->err);
  rc = e->ensure_built();
  if (rc) return serr(s, rc, e->err);
  rc = e->ensure_v();
  if (rc) return serr(s, rc, e->err);
  rc = e->check_status();
  if (rc) return serr(s, rc, e->err);
  // per-system work lists of the pair sum and the reduction
  const size_t nsys = sp.size();
  s->it4_of.assign(nsys, {});
  s->it5_of.assign(nsys, {});
  for (const auto& it : e->L.it4) s->it4_of[it.x].push_back(it);
  for (const auto& it : e->L.it5) s->it5_of[it.x].push_back(it);
  s->pairs_of.assign(nsys, 0.0);
  for (size_t k = 0; k < nsys; ++k) s->pairs_of[k] = (double)ns[k] * (2.0 * ns[k] + sp[k].M);
  int icap = 1, i5cap = 1;
  for (size_t k = 0; k < nsys; ++k) {
    icap = std::max(icap, (int)s->it4_of[k].size());
    i5cap = std::max(i5cap, (int)s->it5_of[k].size());
  }
  // (re)allocate the buffers sized by the resident set
  free_buffers(s);
  s->items_cap = icap;
  s->it5_cap = i5cap;
  int lo = 0, hi = 0;
  SCK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
  if (!s->sA) SCK(cudaStreamCreateWithPriority(&s->sA, cudaStreamNonBlocking, hi));
  s->slots.resize(s->energy_slots);
  for (auto& sl : s->slots) {
    SCK(cudaStreamCreateWithPriority(&sl.st, cudaStreamNonBlocking, lo));
    SCK(cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming));
    SCK(cudaMalloc(&sl.items_d, sizeof(int4) * icap));
    SCK(cudaMalloc(&sl.it5_d, sizeof(int2) * i5cap));
    SCK(cudaMalloc(&sl.sel_d, sizeof(int)));
    SCK(cudaMalloc(&sl.selrng_d, sizeof(int2)));
    SCK(cudaMalloc(&sl.epart_d, 16 * (size_t)i5cap));
    SCK(cudaMalloc(&sl.ctr_d, 2 * sizeof(unsigned int)));
    SCK(cudaMemset(sl.ctr_d, 0, 2 * sizeof(unsigned int)));
    SCK(cudaHostAlloc(&sl.items_h, sizeof(int4) * icap, cudaHostAllocDefault));
    SCK(cudaHostAlloc(&sl.it5_h, sizeof(int2) * i5cap, cudaHostAllocDefault));
    SCK(cudaHostAlloc(&sl.sel_h, sizeof(int), cudaHostAllocDefault));
    SCK(cudaHostAlloc(&sl.selrng_h, sizeof(int2), cudaHostAllocDefault));
    SCK(cudaHostAlloc(&sl.energy_h, 16, cudaHostAllocDefault));
  }
  if (!s->evA) SCK(cudaEventCreateWithFlags(&s->evA, cudaEventDisableTiming));
  const int mb = s->max_batch;
  s->ditems_cap = e->L.ditem_cap;
  s->mitems_cap = e->L.mitem_cap;
  SCK(cudaHostAlloc(&s->dreq_h, sizeof(DeltaReq) * mb, cudaHostAllocDefault));
  SCK(cudaHostAlloc(&s->mreq_h, sizeof(DeltaReq) * mb, cudaHostAllocDefault));
  SCK(cudaHostAlloc(&s->ditems_h, sizeof(int4) * s->ditems_cap, cudaHostAllocDefault));
  SCK(cudaHostAlloc(&s->dranges_h, sizeof(int2) * mb, cudaHostAllocDefault));
  SCK(cudaHostAlloc(&s->mitems_h, sizeof(int2) * s->mitems_cap, cudaHostAllocDefault));
  SCK(cudaHostAlloc(&s->de_h, sizeof(double) * mb, cudaHostAllocDefault));
  SCK(cudaMalloc(&s->mreq_d, sizeof(DeltaReq) * mb));
  SCK(cudaMalloc(&s->mitems_d, sizeof(int2) * s->mitems_cap));
  return HSMA_OK;
}

static int admit(hsma_server_t* s, int* admitted)
{
  size_t used = 0;
  int count = 0;
  for (size_t c = 0; c < s->specs.size(); ++c) {
    s->sys_of[c] = -1;
    if (s->closed[c]) continue;
    if (s->budget == 0 || used + s->footprint[c] <= s->budget) {
      used += s->footprint[c];
      s->sys_of[c] = 0;  // marked resident; rebuild assigns the index
      ++count;
    }
  }
  if (admitted) *admitted = count;
  return rebuild(s);
}

// --- batched move requests ----------------------------------------------------------------
static int launch_moves(hsma_server_t* s, const std::vector<Pending>& batch)
{
  Engine* e = s->e;
  const int nr = (int)batch.size();
  int ni = 0, nacc = 0, nmi = 0;
  for (int r = 0; r < nr; ++r) {
    const hsma_request& q = batch[r].q;
    DeltaReq d;
    d.sys = s->sys_of[q.chain];
    d.k = (int)q.k;
    d.x = q.x[0];
    d.y = q.x[1];
    d.z = q.x[2];
    s->dreq_h[r] = d;
    const hsma::SysDev& sd = e->L.sd[d.sys];
    s->dranges_h[r].x = ni;
    for (int b = 0; b < (sd.n + hsma::kDeltaBlock - 1) / hsma::kDeltaBlock; ++b) s->ditems_h[ni++] = make_int4(r, 0, b, 0);
    for (int b = 0; b < (sd.M + hsma::kDeltaBlock - 1) / hsma::kDeltaBlock; ++b) s->ditems_h[ni++] = make_int4(r, 1, b, 0);
    s->dranges_h[r].y = ni - s->dranges_h[r].x;
    if (q.accept) {
      s->mreq_h[nacc] = d;
      for (int b = 0; b < (sd.M + hsma::kDeltaBlock - 1) / hsma::kDeltaBlock; ++b)
        s->mitems_h[nmi++] = make_int2(nacc, b);
      ++nacc;
    }
  }
  SCK(cudaMemcpyAsync(e->dreq_d, s->dreq_h, sizeof(DeltaReq) * nr, cudaMemcpyHostToDevice, s->sA));
  SCK(cudaMemcpyAsync(e->ditems_d, s->ditems_h, sizeof(int4) * ni, cudaMemcpyHostToDevice, s->sA));
  SCK(cudaMemcpyAsync(e->dreqit_d, s->dranges_h, sizeof(int2) * nr, cudaMemcpyHostToDevice, s->sA));
  hsma::launch_delta(e->sys_d, e->ditems_d, ni, e->dreqit_d, e->dreq_d, nr, e->xyz_d, e->q_d, e->perm_d, e->iperm_d,
                     e->srchi_d, e->srclo_d, e->src64_d, e->surfx_d, e->surfqd_d, e->vsurf_d, e->Mn_d, e->tables(),
                     e->dpart_d, e->de_d, e->ctr_delta_d, e->status_d, s->sA);
  SCK(cudaGetLastError());
  SCK(cudaMemcpyAsync(s->de_h, e->de_d, 8 * nr, cudaMemcpyDeviceToHost, s->sA));
  if (nacc > 0) {
    SCK(cudaMemcpyAsync(s->mreq_d, s->mreq_h, sizeof(DeltaReq) * nacc, cudaMemcpyHostToDevice, s->sA));
    SCK(cudaMemcpyAsync(s->mitems_d, s->mitems_h, sizeof(int2) * nmi, cudaMemcpyHostToDevice, s->sA));
    hsma::launch_move(e->sys_d, s->mitems_d, nmi, s->mreq_d, nacc, e->tables(), e->L.maxP, e->xyz_d, e->q_d,
                      e->Mn_d, e->coef_d, e->coef2_d, e->r0_d, e->surfx_d, e->surfqd_d, e->vsurf_d, 1, e->surfa_d,
                      e->surfb_d, e->surf64a_d, e->surf64b_d, e->iperm_d, e->srchi_d, e->srclo_d, e->src64_d,
                      e->boxes_d, s->sA);
    SCK(cudaGetLastError());
    e->launches += nmi > 0 ? 2 : 1;
    // committed state on the host
    std::lock_guard<std::mutex> lk(s->mu);
    for (int r = 0; r < nr; ++r) {
      const hsma_request& q = batch[r].q;
      if (!q.accept) continue;
      auto& p = s->pos[q.chain];
      p[3 * q.k] = q.x[0];
      p[3 * q.k + 1] = q.x[1];
      p[3 * q.k + 2] = q.x[2];
    }
  }
  e->launches += 1;
  e->pot_ready = false;
  SCK(cudaEventRecord(s->evA, s->sA));
  return HSMA_OK;
}

// Pair evaluations of one pair-sum item (targets x sources, both ways for an off-diagonal
// real/Kelvin item of the FP32 path; a surface point counts once).
static double item_pairs(const hsma::SysDev& d, const int4& it, bool sym)
{
  const bool rk = it.z < d.ncr + d.nck;
  const int cb = it.z < d.ncr ? it.z : it.z - d.ncr;
  const int64_t tbk = sym && rk ? d.chunk : d.tb;
  const double nt = (double)std::min<int64_t>(tbk, (int64_t)d.n - (int64_t)it.y * tbk);
  int64_t ns;
  if (rk)
    ns = std::min<int64_t>(d.chunk, (int64_t)d.n - (int64_t)cb * d.chunk);
  else
    ns = std::min<int64_t>(d.chunk_s, (int64_t)d.M - (int64_t)(it.z - d.ncr - d.nck) * d.chunk_s);
  return nt * (double)std::max<int64_t>(ns, 0) * (sym && rk && cb > it.y ? 2.0 : 1.0);
}

// --- one full-energy request on a slot ------------------------------------------------------
static int launch_energy(hsma_server_t* s, EnergySlot& sl, int chain)
{
  Engine* e = s->e;
  const int sys = s->sys_of[chain];
  const auto& it4 = s->it4_of[sys];
  const auto& it5 = s->it5_of[sys];
  std::copy(it4.begin(), it4.end(), sl.items_h);
  for (size_t k = 0; k < it5.size(); ++k) sl.it5_h[k] = it5[k];
  sl.sel_h[0] = sys;
  sl.selrng_h[0] = make_int2(0, (int)it5.size());
  SCK(cudaMemcpyAsync(sl.items_d, sl.items_h, sizeof(int4) * it4.size(), cudaMemcpyHostToDevice, sl.st));
  SCK(cudaMemcpyAsync(sl.it5_d, sl.it5_h, sizeof(int2) * it5.size(), cudaMemcpyHostToDevice, sl.st));
  SCK(cudaMemcpyAsync(sl.sel_d, sl.sel_h, sizeof(int), cudaMemcpyHostToDevice, sl.st));
  SCK(cudaMemcpyAsync(sl.selrng_d, sl.selrng_h, sizeof(int2), cudaMemcpyHostToDevice, sl.st));
  if (!it4.empty()) {
    const int occ = e->prec == HSMA_FP64 ? e->occ_f64 : e->occ_f32[e->L.cfg];
    const int cap = std::max(1, (int)std::floor(s->sm_frac * e->num_sms * std::max(occ, 1)));
    const int nw = e->L.nw;  // workers per CTA
    const bool sym = e->prec != HSMA_FP64;
    // chunks of consecutive items (the list is longest first) of about kEnergyChunkPairs each,
    // but never fewer items than the capped grid has workers (every launch fills its grid)
    const hsma::SysDev& d = e->L.sd[sys];
    int beg = 0;
    while (beg < (int)it4.size()) {
      int end = beg;
      double w = 0.0;
      while (end < (int)it4.size() &&
             (end - beg < cap * nw || w + item_pairs(d, it4[end], sym) <= kEnergyChunkPairs))
        w += item_pairs(d, it4[end++], sym);
      const int cnt = end - beg;
      const int grid = std::max(1, std::min((cnt + nw - 1) / nw, cap));
      SCK(cudaMemsetAsync(sl.ctr_d, 0, sizeof(unsigned int), sl.st));
      const hsma::PairWork w1{sl.items_d + beg, cnt, sl.ctr_d, std::min(grid * nw, cnt)}, none{nullptr, 0, nullptr, 0};
      if (e->prec == HSMA_FP64)
        hsma::launch_pairs_f64(grid, e->sys_d, w1, none, e->src64_d, e->surf64a_d, e->surf64b_d, e->part64_d, sl.st);
      else
        hsma::launch_pairs_f32(e->L.cfg, grid, e->sys_d, w1, none, e->srchi_d, e->srclo_d, e->surfa_d, e->surfb_d,
                               e->boxes_d, e->part_d, sl.st);
      e->launches += 1;
      beg = end;
    }
  }
  if (!it5.empty()) {
    hsma::launch_reduce(e->sys_d, sl.sel_d, sl.selrng_d, 1, sl.it5_d, (int)it5.size(), e->part_d, e->part64_d, e->prec,
                        e->q_d, e->perm_d, e->r0_d, e->phic_d, e->phir_d, e->phit_d, sl.epart_d, e->energy_d, sl.ctr_d + 1,
                        e->status_d, nullptr, sl.st);
    e->launches += 1;
  }
  SCK(cudaGetLastError());
  SCK(cudaMemcpyAsync(sl.energy_h, e->energy_d + 2 * (size_t)sys, 16, cudaMemcpyDeviceToHost, sl.st));
  SCK(cudaEventRecord(sl.ev, sl.st));
  return HSMA_OK;
}

// --- the request loop -----------------------------------------------------------------------
static void answer(hsma_server_t* s, const Pending& p, int status, double value)
{
  hsma_result r;
  r.id = p.q.id;
  r.status = status;
  r.chain = p.q.chain;
  r.value = value;
  r.t_arrival = p.t_sub;
  r.t_done = now_s() - s->t0;
  r.ticket = p.ticket;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->outbox.push_back(r);
    --s->in_system;
  }
  s->cv_out.notify_all();
}

// Validation of a released request: HSMA_OK or the status it is answered with.
static int check_request(const hsma_server_t* s, const hsma_request& q)
{
  const int nc = (int)s->specs.size();
  if (q.chain < 0 || q.chain >= nc) return HSMA_E_INVALID_ARG;
  if (s->closed[q.chain]) return HSMA_E_BUSY;
  if (q.kind == HSMA_REQ_DELTA) {
    const double a = s->specs[q.chain].a;
    const double r2 = q.x[0] * q.x[0] + q.x[1] * q.x[1] + q.x[2] * q.x[2];
    if (q.k < 0 || q.k >= s->n[q.chain]) return HSMA_E_INVALID_ARG;
    if (!(r2 < a * a) || !std::isfinite(r2)) return HSMA_E_OUTSIDE;
  } else if (q.kind != HSMA_REQ_ENERGY) {
    return HSMA_E_INVALID_ARG;
  }
  return HSMA_OK;
}

static int loop_body(hsma_server_t* s, std::vector<std::deque<Pending>>& fifo, std::vector<Pending>& batch)
{
  Engine* e = s->e;
  SCK(cudaSetDevice(e->device));
  const int nc = (int)s->specs.size();
  std::vector<char> busy(nc, 0);
  bool batch_live = false;
  // admission waiting for the GPU to go idle: chains to evict and to admit
  bool adm_pending = false;
  std::vector<int> adm_out, adm_in;
  std::vector<Pending> incoming;
  for (;;) {
    bool stop = false, drain = true;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      incoming.assign(s->inbox.begin(), s->inbox.end());
      s->inbox.clear();
      stop = s->stop_req;
      drain = s->drain;
    }
    // release: validate, queue per chain
    for (const Pending& p : incoming) {
      const int st = check_request(s, p.q);
      if (st != HSMA_OK)
        answer(s, p, st, 0.0);
      else
        fifo[p.q.chain].push_back(p);
    }
    if (stop && !drain) {
      // cancel what has not started
      for (int c = 0; c < nc; ++c) {
        for (const Pending& p : fifo[c]) answer(s, p, HSMA_E_BUSY, 0.0);
        fifo[c].clear();
      }
    }
    // completions
    if (batch_live) {
      const cudaError_t qe = cudaEventQuery(s->evA);
      if (qe == cudaSuccess) {
        for (size_t i = 0; i < batch.size(); ++i) {
          busy[batch[i].q.chain] = 0;
          answer(s, batch[i], HSMA_OK, s->de_h[i]);
        }
        batch.clear();
        batch_live = false;
      } else if (qe != cudaErrorNotReady) {
        return scuda(s, qe, "move batch");
      }
    }
    for (auto& sl : s->slots) {
      if (!sl.live) continue;
      const cudaError_t qe = cudaEventQuery(sl.ev);
      if (qe == cudaSuccess) {
        busy[sl.chain] = 0;
        sl.live = 0;
        sl.chain = -1;
        answer(s, sl.p, HSMA_OK, sl.energy_h[0]);
      } else if (qe != cudaErrorNotReady) {
        return scuda(s, qe, "energy request");
      }
    }
    int in_flight = batch_live ? 1 : 0;
    for (auto& sl : s->slots) in_flight += sl.live;
    // admission of chains with queued requests that are not resident
    if (!adm_pending) {
      size_t used = 0;
      for (int c = 0; c < nc; ++c)
        if (s->sys_of[c] >= 0) used += s->footprint[c];
      for (int c = 0; c < nc && !adm_pending; ++c) {
        if (fifo[c].empty() || s->sys_of[c] >= 0) continue;
        if (s->budget > 0 && s->footprint[c] > s->budget) {
          for (const Pending& p : fifo[c]) answer(s, p, HSMA_E_BUSY, 0.0);
          fifo[c].clear();
          continue;
        }
        std::vector<int> idle;
        for (int v = 0; v < nc; ++v)
          if (s->sys_of[v] >= 0 && !busy[v] && fifo[v].empty()) idle.push_back(v);
        std::sort(idle.begin(), idle.end(), [&](int x, int y) { return s->last_used[x] < s->last_used[y]; });
        size_t freed = 0;
        std::vector<int> out;
        for (int v : idle) {
          if (s->budget == 0 || used - freed + s->footprint[c] <= s->budget) break;
          out.push_back(v);
          freed += s->footprint[v];
        }
        if (s->budget == 0 || used - freed + s->footprint[c] <= s->budget) {
          adm_pending = true;
          adm_out = out;
          adm_in = {c};
        }
      }
    }
    if (adm_pending && in_flight == 0) {
      for (int v : adm_out) s->sys_of[v] = -1;
      for (int c : adm_in) s->sys_of[c] = 0;  // marked resident; rebuild assigns the index
      adm_pending = false;
      int rc = rebuild(s);
      if (rc) return rc;
    }
    // issue (not while an admission waits for the GPU to go idle)
    if (!adm_pending) {
      if (!batch_live) {
        for (int c = 0; c < nc && (int)batch.size() < s->max_batch; ++c) {
          if (busy[c] || fifo[c].empty() || s->sys_of[c] < 0) continue;
          const Pending& p = fifo[c].front();
          if (p.q.kind != HSMA_REQ_DELTA) continue;
          batch.push_back(p);
          fifo[c].pop_front();
          busy[c] = 1;
          s->last_used[c] = now_s() - s->t0;
        }
        if (!batch.empty()) {
          int rc = launch_moves(s, batch);
          if (rc) return rc;
          batch_live = true;
        }
      }
      for (auto& sl : s->slots) {
        if (sl.live) continue;
        int bc = -1;
        for (int c = 0; c < nc; ++c) {
          if (busy[c] || fifo[c].empty() || s->sys_of[c] < 0) continue;
          const Pending& p = fifo[c].front();
          if (p.q.kind != HSMA_REQ_ENERGY) continue;
          if (bc < 0 || p.t_sub < fifo[bc].front().t_sub) bc = c;
        }
        if (bc < 0) break;
        sl.p = fifo[bc].front();
        fifo[bc].pop_front();
        busy[bc] = 1;
        sl.live = 1;
        sl.chain = bc;
        s->last_used[bc] = now_s() - s->t0;
        int rc = launch_energy(s, sl, bc);
        if (rc) return rc;
      }
    }
    in_flight = batch_live ? 1 : 0;
    for (auto& sl : s->slots) in_flight += sl.live;
    bool queued = false;
    for (int c = 0; c < nc && !queued; ++c) queued = !fifo[c].empty();
    if (stop && in_flight == 0 && !queued) {
      std::lock_guard<std::mutex> lk(s->mu);
      if (s->inbox.empty()) break;
      continue;
    }
    if (in_flight == 0 && !adm_pending) {
      // idle: wait for a submission (or the stop request)
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv_loop.wait_for(lk, std::chrono::milliseconds(2), [&] { return !s->inbox.empty() || s->stop_req; });
    } else {
      std::this_thread::yield();
    }
  }
  // device status of the whole run (a non-finite potential, a bad move)
  SCK(cudaDeviceSynchronize());
  int st = 0;
  SCK(cudaMemcpy(&st, e->status_d, sizeof(int), cudaMemcpyDeviceToHost));
  if (st) {
    cudaMemset(e->status_d, 0, sizeof(int));
    return serr(s, (st & hsma::kStNonFinite) ? HSMA_E_NONFINITE : HSMA_E_OUTSIDE, "device status flagged");
  }
  return HSMA_OK;
}

static void loop_main(hsma_server_t* s)
{
  const int nc = (int)s->specs.size();
  std::vector<std::deque<Pending>> fifo(nc);
  std::vector<Pending> batch;
  int rc = loop_body(s, fifo, batch);
  if (rc) {
    // a CUDA failure ends the loop: everything not answered gets its status
    cudaDeviceSynchronize();
    std::vector<Pending> left(batch.begin(), batch.end());
    for (auto& sl : s->slots)
      if (sl.live) {
        left.push_back(sl.p);
        sl.live = 0;
      }
    for (auto& f : fifo) left.insert(left.end(), f.begin(), f.end());
    {
      std::lock_guard<std::mutex> lk(s->mu);
      left.insert(left.end(), s->inbox.begin(), s->inbox.end());
      s->inbox.clear();
      s->loop_rc = rc;
    }
    for (const Pending& p : left) answer(s, p, rc, 0.0);
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!rc) s->loop_rc = HSMA_OK;
  }
  s->cv_out.notify_all();
}

extern "C" {

int hsma_server_create(int nchains, const double* a, const double* eps1, const double* eps2, const double* kappa,
                       const hsma_params* params, size_t hbm_budget_bytes, int max_batch, int energy_slots,
                       double energy_sm_frac, hsma_server_t** out)
{
  if (!out || nchains <= 0 || !a || !eps1 || !eps2 || !kappa || !params || max_batch < 1 || energy_slots < 1 ||
      !(energy_sm_frac > 0.0) || energy_sm_frac > 1.0)
    return HSMA_E_INVALID_ARG;
  *out = nullptr;
  hsma_server_t* s = new hsma_server_t();
  s->prm = *params;
  s->prm.stream = nullptr;
  for (int c = 0; c < nchains; ++c) {
    SysSpec sp;
    std::string why;
    int rc = hsma::make_spec(a[c], eps1[c], eps2[c], kappa[c], params, &sp, why);
    if (rc) {
      delete s;
      return rc;
    }
    s->specs.push_back(sp);
  }
  s->budget = hbm_budget_bytes;
  s->max_batch = max_batch;
  s->energy_slots = energy_slots;
  s->sm_frac = energy_sm_frac;
  s->e = new Engine();
  s->e->spec = {s->specs[0]};
  int rc = s->e->init(params->device, nullptr, params->precision);
  if (rc) {
    delete s->e;
    delete s;
    return rc;
  }
  *out = s;
  return HSMA_OK;
}

void hsma_server_destroy(hsma_server_t* s)
{
  if (!s) return;
  if (s->running) hsma_server_stop(s, 0);
  if (s->e) cudaSetDevice(s->e->device);
  cudaDeviceSynchronize();
  free_buffers(s);
  if (s->sA) cudaStreamDestroy(s->sA);
  if (s->evA) cudaEventDestroy(s->evA);
  delete s->e;
  delete s;
}

const char* hsma_server_last_error(const hsma_server_t* s) { return s ? s->err.c_str() : "NULL server"; }

int hsma_server_load(hsma_server_t* s, const int64_t* n, const double* xyz, const double* q, int* admitted)
{
  if (!s || !n) return HSMA_E_INVALID_ARG;
  if (s->running) return serr(s, HSMA_E_STATE, "the request loop is running");
  const size_t nc = s->specs.size();
  s->last_used.assign(nc, 0.0);
  s->n.assign(n, n + nc);
  s->pos.assign(nc, {});
  s->chg.assign(nc, {});
  s->footprint.assign(nc, 0);
  s->sys_of.assign(nc, -1);
  s->closed.assign(nc, 0);
  int64_t off = 0;
  for (size_t c = 0; c < nc; ++c) {
    if (n[c] < 0 || n[c] > (int64_t)INT32_MAX / 4) return serr(s, HSMA_E_INVALID_ARG, "bad sizes");
    if (n[c] > 0 && (!xyz || !q)) return serr(s, HSMA_E_INVALID_ARG, "NULL xyz or q");
    const double a = s->specs[c].a;
    for (int64_t i = off; i < off + n[c]; ++i) {
      const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
      if (!(x * x + y * y + z * z < a * a) || !std::isfinite(q[i]))
        return serr(s, HSMA_E_OUTSIDE, "a charge lies outside its cavity");
    }
    s->pos[c].assign(xyz + 3 * off, xyz + 3 * (off + n[c]));
    s->chg[c].assign(q + off, q + off + n[c]);
    // device footprint of the chain on its own
    Engine& e = *s->e;
    e.spec = {s->specs[c]};
    s->footprint[c] = e.make_layout({n[c]}, e.prec == HSMA_FP64 ? 0 : e.choose_config({n[c]})).bytes;
    off += n[c];
  }
  int rc = admit(s, admitted);
  if (rc) return rc;
  s->loaded = true;
  return HSMA_OK;
}

int hsma_server_close_chain(hsma_server_t* s, int c, int* admitted)
{
  if (!s || !s->loaded || c < 0 || c >= (int)s->specs.size()) return serr(s, HSMA_E_INVALID_ARG, "bad chain");
  if (s->running) return serr(s, HSMA_E_STATE, "the request loop is running");
  cudaDeviceSynchronize();
  s->closed[c] = 1;
  return admit(s, admitted);
}

int hsma_server_positions(hsma_server_t* s, int c, double* xyz_out, int64_t n)
{
  if (!s || !s->loaded || c < 0 || c >= (int)s->specs.size() || !xyz_out || n != s->n[c])
    return serr(s, HSMA_E_INVALID_ARG, "bad arguments");
  std::lock_guard<std::mutex> lk(s->mu);
  std::copy(s->pos[c].begin(), s->pos[c].end(), xyz_out);
  return HSMA_OK;
}

int hsma_server_start(hsma_server_t* s)
{
  if (!s) return HSMA_E_INVALID_ARG;
  if (!s->loaded) return serr(s, HSMA_E_STATE, "no chains loaded");
  if (s->running) return serr(s, HSMA_E_STATE, "the request loop is already running");
  SCK(cudaSetDevice(s->e->device));
  SCK(cudaDeviceSynchronize());
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->inbox.clear();
    s->outbox.clear();
    s->in_system = 0;
    s->stop_req = false;
    s->drain = true;
    s->loop_rc = HSMA_OK;
    s->next_ticket = 0;
    s->t0 = now_s();
    s->running = true;
  }
  try {
    s->th = std::thread(loop_main, s);
  } catch (...) {
    s->running = false;
    return serr(s, HSMA_E_STATE, "could not start the request loop thread");
  }
  return HSMA_OK;
}

int hsma_server_submit(hsma_server_t* s, const hsma_request* req, int64_t* ticket)
{
  if (!s || !req) return HSMA_E_INVALID_ARG;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (!s->running || s->stop_req) return HSMA_E_STATE;
    if (s->loop_rc != HSMA_OK) return s->loop_rc;
    if (s->in_system >= s->queue_cap) return HSMA_E_BUSY;
    Pending p;
    p.q = *req;
    p.ticket = s->next_ticket++;
    p.t_sub = now_s() - s->t0;
    s->inbox.push_back(p);
    ++s->in_system;
    if (ticket) *ticket = p.ticket;
  }
  s->cv_loop.notify_one();
  return HSMA_OK;
}

int hsma_server_poll(hsma_server_t* s, hsma_result* out, int max_results, double timeout_s, int* count)
{
  if (!s || !count || max_results < 0 || (max_results > 0 && !out) || !(timeout_s >= 0.0))
    return HSMA_E_INVALID_ARG;
  *count = 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->outbox.empty() && timeout_s > 0.0 && max_results > 0) {
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    s->cv_out.wait_until(lk, deadline, [&] { return !s->outbox.empty() || (!s->running && s->in_system == 0); });
  }
  int k = 0;
  while (k < max_results && !s->outbox.empty()) {
    out[k++] = s->outbox.front();
    s->outbox.pop_front();
  }
  *count = k;
  if (k == 0 && timeout_s > 0.0 && max_results > 0) return HSMA_E_TIMEOUT;
  return HSMA_OK;
}

int hsma_server_stop(hsma_server_t* s, int drain)
{
  if (!s) return HSMA_E_INVALID_ARG;
  if (!s->running) return serr(s, HSMA_E_STATE, "the request loop is not running");
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop_req = true;
    s->drain = drain != 0;
  }
  s->cv_loop.notify_all();
  s->th.join();
  int rc;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->running = false;
    rc = s->loop_rc;
  }
  s->cv_out.notify_all();
  return rc;
}

int hsma_server_run(hsma_server_t* s, int nreq, const hsma_request* reqs, hsma_result* results)
{
  if (!s || nreq < 0 || (nreq > 0 && (!reqs || !results))) return serr(s, HSMA_E_INVALID_ARG, "bad arguments");
  if (!s->loaded) return serr(s, HSMA_E_STATE, "no chains loaded");
  if (s->running) return serr(s, HSMA_E_STATE, "the request loop is running");
  int rc = hsma_server_start(s);
  if (rc) return rc;
  // release order; results[r] answers reqs[r] (found by ticket)
  std::vector<int> order(nreq);
  for (int r = 0; r < nreq; ++r) order[r] = r;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return reqs[x].t_arrival < reqs[y].t_arrival; });
  std::vector<int> of_ticket;
  of_ticket.reserve(nreq);
  const double run0 = now_s();
  const double off = run0 - s->t0;  // run clock = server clock - off
  int next = 0, got = 0;
  std::vector<hsma_result> buf(256);
  while (got < nreq) {
    const double t = now_s() - run0;
    while (next < nreq && reqs[order[next]].t_arrival <= t) {
      int64_t ticket = -1;
      const int sr = hsma_server_submit(s, &reqs[order[next]], &ticket);
      if (sr == HSMA_E_BUSY) break;  // queue full: retry after answers arrive
      if (sr) {
        hsma_server_stop(s, 0);
        return serr(s, sr, "submit failed");
      }
      of_ticket.push_back(order[next]);
      ++next;
    }
    // wait for answers until the next release is due
    const double wait = next < nreq ? std::max(0.0, reqs[order[next]].t_arrival - (now_s() - run0)) : 0.05;
    int cnt = 0;
    const int pr = hsma_server_poll(s, buf.data(), (int)buf.size(), std::min(wait, 0.05), &cnt);
    if (pr != HSMA_OK && pr != HSMA_E_TIMEOUT) {
      hsma_server_stop(s, 0);
      return serr(s, pr, "poll failed");
    }
    if (wait <= 0.0 && cnt == 0) std::this_thread::yield();
    for (int i = 0; i < cnt; ++i) {
      const hsma_result& r = buf[i];
      const int idx = of_ticket[(size_t)r.ticket];
      results[idx] = r;
      results[idx].t_arrival = reqs[idx].t_arrival;
      results[idx].t_done = r.t_done - off;
      ++got;
    }
  }
  return hsma_server_stop(s, 1);
}

}  // extern "C"
